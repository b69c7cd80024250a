// C ABI of the SLLBM library (include/sllbm.h): context, buffers, host-side set-up (velocity set,
// support points, Gauss-Legendre rule, transposed stencils) and dispatch to the kernels.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/sllbm.h"
#include "kernels.h"

using namespace sllbm;

enum StepKernel { kKernelUniform = 0, kKernelGather = 1, kKernelPlainF64 = 2, kKernelMapped = 3, kKernelQ9 = 4 };
constexpr int kXferChunks = 5;   // host transfers move the state in this many plane groups
// sllbm_step calls of at least kGraphMinSteps steps replay a graph on grids whose state buffer is at
// most kGraphMaxStateBytes: L2-resident steps are bound by launch overhead.  (On large grids the
// direct launches are as fast, or faster where the fix-up gather overlaps the fused kernel on
// its side stream: 0.908 against 0.958 ms a step on the 3073^2 Riemann grid.)
constexpr int kGraphMinSteps = 4;
constexpr size_t kGraphMaxStateBytes = size_t(64) << 20;

struct sllbm_ctx {
  sllbm_grid_desc g;
  sllbm_params p;
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, npop = 2, P = 0, store = kStoreF32, elem = 4;
  int nq1 = kQ1, nq = kQ;                // velocity set: D2Q25, or D2Q9 (nq1 = 3, nq = 9)
  long long nv = 0;
  // State layout (StepArgs): value (pop, i, y, x) at i * plane_stride + pop * ps + y * pitch +
  // x * xs from the interior origin; pitchv vertices per row.  FP32/BF16: (f, g) interleaved
  // (xs = 2, ps = 1); FP64, and every D2Q9 state: planar (xs = 1, ps = nq planes).
  int pitchv = 0, pitch = 0, xs = 1;
  size_t plane_stride = 0;
  ptrdiff_t ps = 0;
  void* dense = nullptr;                 // dense staging state for host transfers (on demand)
  cudaStream_t xfer = nullptr;           // copy stream of the host transfers (on demand)
  cudaStream_t side = nullptr;           // fix-up launches beside the fused kernel (on demand)
  cudaEvent_t side_ev[2] = {};
  cudaGraphExec_t step_graph = nullptr;  // two steps (state 0 -> 1 -> 0), captured on demand
  bool graph_off = false;                // the stream cannot be captured: steps launch directly
  cudaEvent_t xev[kXferChunks + 1] = {};
  AxisK ax{}, ay{};
  MapK map{};
  Consts cs{};
  CollideK cp{};
  void* state[2] = {nullptr, nullptr};   // interior origins of the two state buffers
  void* alloc[2] = {nullptr, nullptr};   // allocation starts (ghost cells included)
  int gx = 8, gy = 4, gxr = 0, gyb = 20, rows_alloc = 0;
  GhostK ghost{};
  int cur = 0;
  bool precomputed = false, initialized = false;
  int kernel = kKernelGather;
  int q9_tma = 0;                        // D2Q9 FP32/BF16 uniform: the TMA-staged kernel
  // uniform tables
  int *offx = nullptr, *offy = nullptr;
  float *wx = nullptr, *wy = nullptr;
  double *wx64 = nullptr, *wy64 = nullptr;
  int offx_lo = 0, offx_hi = 0, offy_lo = 0, offy_hi = 0;
  UniformTables ut{};
  unsigned char *std_x = nullptr, *std_y = nullptr;
  int* fix_list = nullptr;       // vertices the fused kernels leave to the gather kernel
  long long n_fix = 0;
  // mapped-grid tiles
  MappedTables mt{};
  uint32_t* mrec = nullptr;
  int2* morg = nullptr;
  unsigned char* mok = nullptr;
  // per-(velocity, vertex) descriptors
  int *dcx = nullptr, *dcy = nullptr;
  float *dr = nullptr, *ds = nullptr;
  double *dr64 = nullptr, *ds64 = nullptr;
  // diagnostics
  double* A = nullptr;
  double* partials = nullptr;
  double* sums = nullptr;
  int* flag = nullptr;
  // adjoint
  bool transposed = false;
  float* mu = nullptr;                                  // J_C^T pairs (two-pass and mapped S^T)
  int mu_g = 0, mu_pitch = 0, mu_rows = 0;              // ghost-padded layout of mu (one-pass S^T)
  int *tx_col = nullptr, *ty_col = nullptr, tkw = 0;   // fixed-width transposed stencils
  int thalo = 0;                                        // their largest source-target offset
  float *tx_dense = nullptr, *ty_dense = nullptr;       // dense by offset (one-pass S^T)
  int thalo_k = 0, tdw = 0;                             // its halo and row width
  int *tx_deg = nullptr, *ty_deg = nullptr;
  float2* atmp = nullptr;                               // between the x and y passes of S^T
  float *tx_w = nullptr, *ty_w = nullptr;
  long long* tm_ptr = nullptr;
  int* tm_col = nullptr;
  float* tm_w = nullptr;
  std::vector<void*> allocations;
  std::string err;
};

// ------------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------------
static sllbm_status fail(sllbm_ctx* c, sllbm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

static sllbm_status cuda_fail(sllbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, SLLBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(ctx, call)                                 \
  do {                                                      \
    cudaError_t _e = (call);                                \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call); \
  } while (0)

template <typename T>
static sllbm_status dalloc(sllbm_ctx* c, T** ptr, size_t count) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, SLLBM_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                      " bytes failed: " + cudaGetErrorString(e));
  }
  c->allocations.push_back(p);
  *ptr = static_cast<T*>(p);
  return SLLBM_OK;
}

#define TRY(call)                          \
  do {                                     \
    sllbm_status _s = (call);              \
    if (_s != SLLBM_OK) return _s;         \
  } while (0)

// D1Q5 abscissae and weights in Table I order (or the D1Q3 ones, 0, +sqrt3, -sqrt3 with
// 2/3, 1/6, 1/6, for the D2Q9 set, the rest of the arrays zero); he[k][a] = He_k(xi_a) / k! by
// the recurrence He_{k+1}(x) = x He_k(x) - k He_{k-1}(x).
static void build_consts(Consts& cs, int velset) {
  cs = Consts{};
  const double s10 = sqrt(10.0);
  const double sm = sqrt(5.0 - s10), lg = sqrt(5.0 + s10);
  const double xi5[5] = {0.0, sm, lg, -sm, -lg};
  const double w5[5] = {8.0 / 15.0, (7.0 + 2.0 * s10) / 60.0, (7.0 - 2.0 * s10) / 60.0,
                        (7.0 + 2.0 * s10) / 60.0, (7.0 - 2.0 * s10) / 60.0};
  const double xi3[5] = {0.0, sqrt(3.0), -sqrt(3.0), 0.0, 0.0};
  const double w3[5] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 0.0, 0.0};
  const bool q9 = velset == SLLBM_VEL_D2Q9;
  const double* xi = q9 ? xi3 : xi5;
  const double* w = q9 ? w3 : w5;
  cs.nq1 = q9 ? 3 : 5;
  for (int a = 0; a < cs.nq1; ++a) {
    cs.xi[a] = xi[a];
    cs.w[a] = w[a];
    double hm1 = 0.0, h = 1.0, fact = 1.0;
    for (int k = 0; k < 5; ++k) {
      if (k > 0) fact *= k;
      cs.he[k][a] = h / fact;
      const double hn = xi[a] * h - k * hm1;
      hm1 = h;
      h = hn;
    }
    cs.xif[a] = (float)xi[a];
    cs.wf[a] = (float)w[a];
    for (int k = 0; k < 5; ++k) {
      cs.hef[k][a] = (float)cs.he[k][a];
      cs.whf[k][a] = (float)(cs.w[a] * cs.he[k][a]);
    }
  }
  cs.inv_xi1f = (float)(1.0 / xi[1]);
  cs.xi1sqf = (float)(xi[1] * xi[1]);
}

static void build_axis(AxisK& ax, int n_cells, int p, double lo, double hi, int periodic, int nodes) {
  ax.n_cells = n_cells;
  ax.p = p;
  ax.periodic = periodic;
  ax.nv = periodic ? n_cells * p : n_cells * p + 1;
  ax.lo = lo;
  ax.hi = hi;
  ax.len = hi - lo;
  ax.hc = (hi - lo) / n_cells;
  const double pi = 3.141592653589793238462643383279502884;
  for (int k = 0; k < 5; ++k) ax.nodes[k] = 0.0;
  for (int k = 0; k <= p; ++k)  // Gauss-Lobatto-Chebyshev points (Sec. II.E) or equidistant
    ax.nodes[k] = nodes == SLLBM_NODES_GLC ? 0.5 * (1.0 - cos(k * pi / p)) : (double)k / p;
}

// Gauss-Legendre rule with n points on [0, 1] (Newton on the Legendre recurrence).
static void gauss_legendre01(int n, double* x, double* w) {
  const double pi = 3.141592653589793238462643383279502884;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2)P'^2) on [-1,1], halved for [0,1]
  }
}

static StepArgs step_args(sllbm_ctx* c, const void* src, void* dst) {
  StepArgs a{};
  a.src = src;
  a.dst = dst;
  a.nx = c->nx;
  a.ny = c->ny;
  a.pitch = c->pitch;
  a.periodic_x = c->ax.periodic;
  a.periodic_y = c->ay.periodic;
  a.P = c->P;
  a.nv = c->nv;
  a.plane_stride = c->plane_stride;
  a.xs = c->xs;
  a.ps = c->ps;
  a.offx = c->offx;
  a.offy = c->offy;
  a.wx = c->wx;
  a.wy = c->wy;
  a.wx64 = c->wx64;
  a.wy64 = c->wy64;
  a.dcx = c->dcx;
  a.dcy = c->dcy;
  a.dr = c->dr;
  a.ds = c->ds;
  a.dr64 = c->dr64;
  a.ds64 = c->ds64;
  for (int k = 0; k < 5; ++k) {
    a.nodes[k] = c->ax.nodes[k];
    a.nodesf[k] = (float)c->ax.nodes[k];
  }
  a.cs = c->cs;
  a.cp = c->cp;
  a.flag = c->flag;
  a.mapped = (c->map.kind != SLLBM_MAP_IDENTITY) || (c->kernel == kKernelGather && c->dcx != nullptr);
  a.offx_min = c->offx_lo;
  a.offx_max = c->offx_hi;
  a.offy_min = c->offy_lo;
  a.offy_max = c->offy_hi;
  a.ghost = c->ghost;
  a.q9_tma = c->q9_tma;
  a.gx = c->gx;
  a.gy = c->gy;
  a.rows_alloc = c->rows_alloc;
  return a;
}

static GeomArgs geom_args(sllbm_ctx* c) {
  GeomArgs g{};
  g.ax = c->ax;
  g.ay = c->ay;
  g.map = c->map;
  g.cs = c->cs;
  g.dt = c->p.dt;
  g.nx = c->nx;
  g.ny = c->ny;
  g.nv = c->nv;
  g.flag = c->flag;
  return g;
}

// Cell-periodic pattern of the per-axis tables of a uniform grid (read by step_uniform.cu):
// taken from a cell in the middle of each axis; a vertex "follows the pattern" when its offset
// and weights match those of its local node for all five components.  The fused kernel writes
// only vertices that follow the pattern on both axes; the others go to the gather kernel.
static sllbm_status axis_pattern(sllbm_ctx* c, const AxisK& ax, const int* off_dev, const double* w_dev,
                                 bool is_y, std::vector<unsigned char>& stdv, bool* ok) {
  const int n = ax.nv, P = c->P;
  std::vector<int> off((size_t)kQ1 * n);
  std::vector<double> w((size_t)kQ1 * n * (P + 1));
  CUDA_TRY(c, cudaMemcpyAsync(off.data(), off_dev, off.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(w.data(), w_dev, w.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *ok = ax.n_cells >= 3;
  const int jref0 = (ax.n_cells / 2) * P;
  for (int comp = 0; comp < kQ1 && *ok; ++comp)
    for (int k = 0; k < P; ++k) {
      const int j = jref0 + k;
      const int d = off[(size_t)comp * n + j];
      if (d < -P || d > 0) { *ok = false; break; }   // taps must stay within the band [-P, P]
      const double* wj = &w[((size_t)comp * n + j) * (P + 1)];
      if (is_y) {
        c->ut.dy_pat[comp][k] = d;
        for (int al = 0; al <= P; ++al) c->ut.wy_pat[comp][k][al] = wj[al];
      } else {
        c->ut.dx_pat[comp][k] = d;
        for (int al = 0; al <= P; ++al) c->ut.wx_pat[comp][k][al] = wj[al];
      }
    }
  stdv.assign(n, 1);
  for (int j = 0; j < n && *ok; ++j) {
    const int k = j % P;
    for (int comp = 0; comp < kQ1; ++comp) {
      const int d = off[(size_t)comp * n + j];
      const double* wj = &w[((size_t)comp * n + j) * (P + 1)];
      const int dref = off[(size_t)comp * n + jref0 + k];
      const double* wr = &w[((size_t)comp * n + jref0 + k) * (P + 1)];
      bool same = (d == dref);
      for (int al = 0; al <= P && same; ++al) same = fabs(wj[al] - wr[al]) <= 1e-6;
      if (!same) stdv[j] = 0;
    }
  }
  return SLLBM_OK;
}

static sllbm_status build_uniform_pattern(sllbm_ctx* c) {
  c->ut.valid = false;
  // 16-byte staging chunks must not straddle the periodic seam, and tiles need a few cells
  if (c->xs != 2 || (c->ax.periodic && c->nx % 4 != 0)) return SLLBM_OK;
  std::vector<unsigned char> sx, sy;
  bool okx = false, oky = false;
  TRY(axis_pattern(c, c->ax, c->offx, c->wx64, false, sx, &okx));
  TRY(axis_pattern(c, c->ay, c->offy, c->wy64, true, sy, &oky));
  if (!okx || !oky) return SLLBM_OK;
  // The fused kernel takes each stencil as a whole cell, on both axes: start offset -l at local
  // node l, or -P at node 0 (a departure into the cell before).  Anything else goes to the
  // gather path.
  for (int comp = 0; comp < kQ1; ++comp)
    for (int k = 0; k < c->P; ++k) {
      const int dy = c->ut.dy_pat[comp][k], dx = c->ut.dx_pat[comp][k];
      if (k == 0 ? (dy != 0 && dy != -c->P) : dy != -k) return SLLBM_OK;
      if (k == 0 ? (dx != 0 && dx != -c->P) : dx != -k) return SLLBM_OK;
    }
  if (!c->std_x) {
    TRY(dalloc(c, &c->std_x, (size_t)c->nx));
    TRY(dalloc(c, &c->std_y, (size_t)c->ny));
  }
  CUDA_TRY(c, cudaMemcpy(c->std_x, sx.data(), sx.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->std_y, sy.data(), sy.size(), cudaMemcpyHostToDevice));
  std::vector<int> fix;
  for (int iy = 0; iy < c->ny; ++iy)
    for (int ix = 0; ix < c->nx; ++ix)
      if (!sx[ix] || !sy[iy]) fix.push_back(iy * c->nx + ix);
  c->n_fix = (long long)fix.size();
  if (!fix.empty()) {
    TRY(dalloc(c, &c->fix_list, fix.size()));
    CUDA_TRY(c, cudaMemcpy(c->fix_list, fix.data(), fix.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  c->ut.std_x = c->std_x;
  c->ut.std_y = c->std_y;
  c->ut.gx = c->gx;
  c->ut.gy = c->gy;
  c->ut.rows_alloc = c->rows_alloc;
  c->ut.valid = true;
  return SLLBM_OK;
}

// Tail-weight polynomials of the Lagrange basis on the axis nodes: W_alpha(r) = sum_{beta >= alpha}
// psi_beta(r), expanded in t = r - 1/2 (FP64 expansion, FP32 coefficients).
static void tail_weight_polys(const double* nodes, int P, float wc[4][5]) {
  for (int al = 0; al < 4; ++al)
    for (int j = 0; j < 5; ++j) wc[al][j] = 0.f;
  double tails[5][5] = {};
  for (int b = 0; b <= P; ++b) {
    double poly[5] = {1.0, 0, 0, 0, 0};   // coefficients in t, low order first
    int deg = 0;
    for (int m = 0; m <= P; ++m) {
      if (m == b) continue;
      const double c0 = -(nodes[m] - 0.5), inv = 1.0 / (nodes[b] - nodes[m]);
      double next[5] = {0, 0, 0, 0, 0};
      for (int j = 0; j <= deg; ++j) {
        next[j + 1] += poly[j] * inv;
        next[j] += poly[j] * c0 * inv;
      }
      ++deg;
      for (int j = 0; j < 5; ++j) poly[j] = next[j];
    }
    for (int al = 1; al <= b; ++al)
      for (int j = 0; j <= P; ++j) tails[al][j] += poly[j];
  }
  for (int al = 1; al <= P; ++al)
    for (int j = 0; j <= P; ++j) wc[al - 1][j] = (float)tails[al][j];
}

// Staged windows of the fused mapped-grid kernel (read by step_mapped.cu).  Per tile of 32 x 8
// vertices and velocity plane: the bounding box of the stencils (cell start nodes, unwrapped
// across periodic seams relative to the vertex), its origin rounded down to a 16-byte boundary.
// The window size is the largest box over all tiles; a tile whose stencils leave the ghost-cell
// layout, or whose box exceeds the window limit, goes to the gather kernel.
static sllbm_status build_mapped_tiles(sllbm_ctx* c) {
  c->mt.valid = false;
  if (c->xs != 2) return SLLBM_OK;
  const int P = c->P, nx = c->nx, ny = c->ny;
  const long long nv = c->nv;
  const size_t n = (size_t)kQ * nv;
  std::vector<int> cx(n), cy(n);
  std::vector<float> rr(n), ss(n);
  CUDA_TRY(c, cudaMemcpyAsync(cx.data(), c->dcx, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(cy.data(), c->dcy, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(rr.data(), c->dr, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(ss.data(), c->ds, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const int tiles_x = (nx + kMappedTileX - 1) / kMappedTileX, tiles_y = (ny + kMappedTileY - 1) / kMappedTileY;
  const int ntiles = tiles_x * tiles_y;
  const int A = (c->store == kStoreBF16) ? 4 : 2;      // pairs per 16 bytes
  auto unwrap = [](int node, int vert, int nvert, bool periodic) {
    if (periodic) {
      if (node - vert > nvert / 2) node -= nvert;
      if (node - vert < -nvert / 2) node += nvert;
    }
    return node;
  };
  const int xlo = -c->gx, xhi = nx + c->gxr, ylo = -c->gy, yhi = ny + c->gyb;
  std::vector<int2> org((size_t)ntiles * kQ);
  std::vector<int> extx((size_t)ntiles * kQ), exty((size_t)ntiles * kQ);
  std::vector<unsigned char> ok(ntiles, 1);
  int bw = 0, bh = 0;
  for (int t = 0; t < ntiles; ++t) {
    const int x0 = (t % tiles_x) * kMappedTileX, y0 = (t / tiles_x) * kMappedTileY;
    for (int i = 0; i < kQ; ++i) {
      int mnx = 1 << 30, mxx = -(1 << 30), mny = 1 << 30, mxy = -(1 << 30);
      for (int y = y0; y < std::min(y0 + kMappedTileY, ny); ++y)
        for (int x = x0; x < std::min(x0 + kMappedTileX, nx); ++x) {
          const size_t d = (size_t)i * nv + (size_t)y * nx + x;
          const int X = unwrap(cx[d] * P, x, nx, c->ax.periodic), Y = unwrap(cy[d] * P, y, ny, c->ay.periodic);
          mnx = std::min(mnx, X);
          mxx = std::max(mxx, X);
          mny = std::min(mny, Y);
          mxy = std::max(mxy, Y);
        }
      if (mnx < xlo || mxx + P >= xhi || mny < ylo || mxy + P >= yhi) ok[t] = 0;
      const int ox = mnx - (((mnx + c->gx) % A) + A) % A;
      org[(size_t)t * kQ + i] = make_int2(ox, mny);
      extx[(size_t)t * kQ + i] = mxx + P + 1 - ox;
      exty[(size_t)t * kQ + i] = mxy + P + 1 - mny;
      if (ok[t]) {
        bw = std::max(bw, extx[(size_t)t * kQ + i]);
        bh = std::max(bh, exty[(size_t)t * kQ + i]);
      }
    }
  }
  bw = (bw + A - 1) / A * A;
  // two CTAs per SM: at most ~110 KB of staging per CTA; a tile that needs more goes to the
  // gather kernel
  const size_t limit = 110 * 1024;
  while (bw > A && mapped_smem_bytes(bw, bh, c->store) > limit) {
    if (bw >= 2 * bh) bw -= A; else --bh;
  }
  if (bw < P + 1 || bh < P + 1 || 2 * bw > 256 || bh > 256) return SLLBM_OK;
  for (int t = 0; t < ntiles; ++t)
    for (int i = 0; i < kQ && ok[t]; ++i)
      if (extx[(size_t)t * kQ + i] > bw || exty[(size_t)t * kQ + i] > bh) ok[t] = 0;
  // records [field][plane][row][column]: rows up to the last tile, columns up to dpitch
  const int dpitch = tiles_x * kMappedTileX, drows = tiles_y * kMappedTileY;
  const size_t fstride = (size_t)kQ * drows * dpitch;
  std::vector<uint32_t> rec(3 * fstride, 0u);
  std::vector<int> fix;
  for (int t = 0; t < ntiles; ++t) {
    const int x0 = (t % tiles_x) * kMappedTileX, y0 = (t / tiles_x) * kMappedTileY;
    for (int y = y0; y < std::min(y0 + kMappedTileY, ny); ++y)
      for (int x = x0; x < std::min(x0 + kMappedTileX, nx); ++x) {
        if (!ok[t]) {
          fix.push_back(y * nx + x);
          continue;
        }
        for (int i = 0; i < kQ; ++i) {
          const size_t d = (size_t)i * nv + (size_t)y * nx + x;
          const int2 o = org[(size_t)t * kQ + i];
          const int X = unwrap(cx[d] * P, x, nx, c->ax.periodic), Y = unwrap(cy[d] * P, y, ny, c->ay.periodic);
          const size_t e = ((size_t)i * drows + y) * dpitch + x;
          rec[e] = ((uint32_t)(Y - o.y) << 16) | (uint32_t)(X - o.x);
          memcpy(&rec[fstride + e], &rr[d], 4);
          memcpy(&rec[2 * fstride + e], &ss[d], 4);
        }
      }
  }
  if (fix.size() == (size_t)nv) return SLLBM_OK;   // nothing for the fused kernel
  if (!c->mrec) {
    TRY(dalloc(c, &c->mrec, rec.size()));
    TRY(dalloc(c, &c->morg, org.size()));
    TRY(dalloc(c, &c->mok, (size_t)ntiles));
  }
  CUDA_TRY(c, cudaMemcpy(c->mrec, rec.data(), rec.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->morg, org.data(), org.size() * sizeof(int2), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->mok, ok.data(), ok.size(), cudaMemcpyHostToDevice));
  c->n_fix = (long long)fix.size();
  if (!fix.empty()) {
    TRY(dalloc(c, &c->fix_list, fix.size()));
    CUDA_TRY(c, cudaMemcpy(c->fix_list, fix.data(), fix.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  c->mt.rec = c->mrec;
  c->mt.dpitch = dpitch;
  c->mt.org = c->morg;
  c->mt.tile_ok = c->mok;
  c->mt.bw = bw;
  c->mt.bh = bh;
  c->mt.gx = c->gx;
  c->mt.gy = c->gy;
  c->mt.rows_alloc = c->rows_alloc;
  tail_weight_polys(c->ax.nodes, P, c->mt.wc);
  c->mt.valid = true;
  return SLLBM_OK;
}

// Dense [npop][25][ny][nx] <-> the internal layout.  Host transfers go through the dense staging
// buffer and the conversion kernel in kXferChunks plane groups: the copy of one group (on the
// context's copy stream) overlaps the conversion of the previous one (on its compute stream).
static cudaError_t convert_state(sllbm_ctx* c, const void* src, void* dst, bool to_internal,
                                 int plane0, int nplanes) {
  return launch_state_convert(src, dst, to_internal, c->elem, plane0, nplanes, c->nq, c->nx, c->ny, c->pitch,
                              c->plane_stride, c->xs, c->ps, c->stream);
}

// Interleaved (f, g) pairs convert by velocity plane, both populations at once.
static bool pair_layout(const sllbm_ctx* c) { return c->xs == 2 && c->ps == 1 && c->ny <= 65535; }

static cudaError_t convert_pairs(sllbm_ctx* c, const void* src, void* dst, bool to_internal, int i0, int ni) {
  return launch_pair_convert(src, dst, to_internal, c->elem, i0, ni, c->npop, c->nq, c->nx, c->ny, c->pitch,
                             c->plane_stride, c->stream);
}

static size_t dense_bytes(const sllbm_ctx* c) { return (size_t)c->npop * c->nq * c->nv * c->elem; }

// Dense [npop][nq][ny][nx] state (host or device) <-> the internal layout.  Host transfers go in
// kXferChunks groups of planes on a copy stream, each group's conversion on the compute stream
// overlapping the next group's copy.  With (f, g) pairs a group is a range of velocity planes
// with both populations (one copy per population), converted pair by pair.
static sllbm_status copy_state(sllbm_ctx* c, void* dst, const void* src, bool to_internal, cudaMemcpyKind kind) {
  const bool pairs = pair_layout(c);
  const int planes = c->npop * c->nq;
  if (kind == cudaMemcpyDeviceToDevice) {
    if (pairs)
      CUDA_TRY(c, convert_pairs(c, src, dst, to_internal, 0, c->nq));
    else
      CUDA_TRY(c, convert_state(c, src, dst, to_internal, 0, planes));
    return SLLBM_OK;
  }
  if (!c->dense) {
    char* p = nullptr;
    TRY(dalloc(c, &p, dense_bytes(c)));
    c->dense = p;
  }
  if (!c->xfer) {
    CUDA_TRY(c, cudaStreamCreateWithFlags(&c->xfer, cudaStreamNonBlocking));
    for (int k = 0; k <= kXferChunks; ++k) CUDA_TRY(c, cudaEventCreateWithFlags(&c->xev[k], cudaEventDisableTiming));
  }
  const size_t plane_bytes = (size_t)c->nv * c->elem;
  const int units = pairs ? c->nq : planes;   // chunked unit: velocity plane (pairs) or dense plane
  const int copies = pairs ? c->npop : 1;     // host copies per chunk
  const size_t pop_bytes = (size_t)c->nq * plane_bytes;
  // the copy stream starts after the work already queued on the compute stream
  CUDA_TRY(c, cudaEventRecord(c->xev[kXferChunks], c->stream));
  CUDA_TRY(c, cudaStreamWaitEvent(c->xfer, c->xev[kXferChunks], 0));
  char* dense = static_cast<char*>(c->dense);
  for (int k = 0; k < kXferChunks; ++k) {
    const int p0 = units * k / kXferChunks, np = units * (k + 1) / kXferChunks - p0;
    if (np == 0) continue;
    if (to_internal) {
      for (int q = 0; q < copies; ++q) {
        const size_t off = q * pop_bytes + p0 * plane_bytes;
        CUDA_TRY(c, cudaMemcpyAsync(dense + off, static_cast<const char*>(src) + off, np * plane_bytes,
                                    cudaMemcpyHostToDevice, c->xfer));
      }
      CUDA_TRY(c, cudaEventRecord(c->xev[k], c->xfer));
      CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->xev[k], 0));
      if (pairs)
        CUDA_TRY(c, convert_pairs(c, dense, dst, true, p0, np));
      else
        CUDA_TRY(c, convert_state(c, dense, dst, true, p0, np));
    } else {
      if (pairs)
        CUDA_TRY(c, convert_pairs(c, src, dense, false, p0, np));
      else
        CUDA_TRY(c, convert_state(c, src, dense, false, p0, np));
      CUDA_TRY(c, cudaEventRecord(c->xev[k], c->stream));
      CUDA_TRY(c, cudaStreamWaitEvent(c->xfer, c->xev[k], 0));
      for (int q = 0; q < copies; ++q) {
        const size_t off = q * pop_bytes + p0 * plane_bytes;
        CUDA_TRY(c, cudaMemcpyAsync(static_cast<char*>(dst) + off, dense + off, np * plane_bytes,
                                    cudaMemcpyDeviceToHost, c->xfer));
      }
    }
  }
  // the compute stream resumes after the last copy (so that synchronising it covers the transfer,
  // and the staging buffer is not reused before the copies out of it are done)
  CUDA_TRY(c, cudaEventRecord(c->xev[kXferChunks], c->xfer));
  CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->xev[kXferChunks], 0));
  return SLLBM_OK;
}

static cudaError_t fill_ghosts(sllbm_ctx* c) {
  if (!c->ghost.on) return cudaSuccess;
  // interleaved layout: an (f, g) pair moves as one element of twice the size
  if (c->xs == 2)
    return launch_ghost_fill(c->state[c->cur], 2 * c->elem, c->plane_stride / 2, c->pitchv, kQ,
                             c->ghost, c->stream);
  return launch_ghost_fill(c->state[c->cur], c->elem, c->plane_stride, c->pitch, c->npop * c->nq,
                           c->ghost, c->stream);
}

// ------------------------------------------------------------------------------------------
// API
// ------------------------------------------------------------------------------------------
extern "C" {

const char* sllbm_status_string(sllbm_status s) {
  switch (s) {
    case SLLBM_OK: return "ok";
    case SLLBM_ERR_ARG: return "invalid argument";
    case SLLBM_ERR_CUDA: return "CUDA error";
    case SLLBM_ERR_OOM: return "out of memory";
    case SLLBM_ERR_STATE: return "call order (precompute/init missing)";
    case SLLBM_ERR_NEWTON: return "Newton inversion of the grid map failed";
    case SLLBM_ERR_UNSTABLE: return "unstable: non-positive or non-finite density/temperature";
    case SLLBM_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* sllbm_last_error(const sllbm_ctx* c) { return c ? c->err.c_str() : "null context"; }

sllbm_status sllbm_destroy(sllbm_ctx* c) {
  if (!c) return SLLBM_ERR_ARG;
  if (c->step_graph) {
    cudaStreamSynchronize(c->stream);
    cudaGraphExecDestroy(c->step_graph);
  }
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
    for (int k = 0; k < 2; ++k)
      if (c->side_ev[k]) cudaEventDestroy(c->side_ev[k]);
  }
  if (c->xfer) {
    cudaStreamSynchronize(c->xfer);
    cudaStreamDestroy(c->xfer);
    for (int k = 0; k <= kXferChunks; ++k)
      if (c->xev[k]) cudaEventDestroy(c->xev[k]);
  }
  for (void* p : c->allocations) cudaFree(p);
  delete c;
  return SLLBM_OK;
}

sllbm_status sllbm_create(const sllbm_grid_desc* g, const sllbm_params* p, void* stream, sllbm_ctx** out) {
  if (!g || !p || !out) return SLLBM_ERR_ARG;
  *out = nullptr;
  if (g->order < 1 || g->order > 4) return SLLBM_ERR_UNSUPPORTED;
  if (p->velset != SLLBM_VEL_D2Q25_HERMITE && p->velset != SLLBM_VEL_D2Q9) return SLLBM_ERR_UNSUPPORTED;
  if (g->nx_cells < 1 || g->ny_cells < 1 || !(g->x1 > g->x0) || !(g->y1 > g->y0)) return SLLBM_ERR_ARG;
  if ((g->bc_x != SLLBM_BC_PERIODIC && g->bc_x != SLLBM_BC_ZERO_GRADIENT) ||
      (g->bc_y != SLLBM_BC_PERIODIC && g->bc_y != SLLBM_BC_ZERO_GRADIENT))
    return SLLBM_ERR_ARG;
  if (g->nodes != SLLBM_NODES_GLC && g->nodes != SLLBM_NODES_EQUIDISTANT) return SLLBM_ERR_ARG;
  if (g->map != SLLBM_MAP_IDENTITY && g->map != SLLBM_MAP_SINE) return SLLBM_ERR_ARG;
  if (p->prec != SLLBM_PREC_F32 && p->prec != SLLBM_PREC_BF16_STORE && p->prec != SLLBM_PREC_F64_PLAIN)
    return SLLBM_ERR_ARG;
  if (!(p->dt > 0.0) || !(p->tau > 0.5) || !(p->cv >= 1.0) || p->T0 != 1.0) return SLLBM_ERR_ARG;
  if (!(p->pr >= 0.0) || !(p->pr < 1e6)) return SLLBM_ERR_ARG;   // NaN, negative or absurd
  if (p->isothermal != 0 && (p->isothermal != 1 || p->cv != 1.0)) return SLLBM_ERR_ARG;
  // D2Q9 carries the isothermal configuration only (Sec. III.A), with plain BGK
  if (p->velset == SLLBM_VEL_D2Q9 && (p->isothermal != 1 || (p->pr != 0.0 && p->pr != 1.0)))
    return SLLBM_ERR_UNSUPPORTED;
  if ((long long)g->nx_cells * g->order > (1 << 20) || (long long)g->ny_cells * g->order > (1 << 20))
    return SLLBM_ERR_UNSUPPORTED;
  sllbm_ctx* c = new (std::nothrow) sllbm_ctx();
  if (!c) return SLLBM_ERR_OOM;
  c->g = *g;
  c->p = *p;
  c->stream = static_cast<cudaStream_t>(stream);
  c->P = g->order;
  build_consts(c->cs, p->velset);
  c->nq1 = c->cs.nq1;
  c->nq = c->nq1 * c->nq1;
  build_axis(c->ax, g->nx_cells, g->order, g->x0, g->x1, g->bc_x == SLLBM_BC_PERIODIC, g->nodes);
  build_axis(c->ay, g->ny_cells, g->order, g->y0, g->y1, g->bc_y == SLLBM_BC_PERIODIC, g->nodes);
  c->map.kind = g->map;
  c->map.a = g->map_param[0];
  c->nx = c->ax.nv;
  c->ny = c->ay.nv;
  c->nv = (long long)c->nx * c->ny;
  c->npop = (p->cv == 1.0) ? 1 : 2;
  c->cp.omega = 1.0 / p->tau;
  c->cp.cv = p->cv;
  c->cp.K = 2.0 * p->cv - 2.0;
  c->cp.omegaf = (float)c->cp.omega;
  c->cp.cvf = (float)p->cv;
  c->cp.Kf = (float)c->cp.K;
  c->cp.inv2cvf = (float)(0.5 / p->cv);
  c->cp.npop = c->npop;
  c->cp.iso = p->isothermal;
  {
    const double pr = (p->pr == 0.0) ? 1.0 : p->pr;
    const double tau_pr = (p->tau - 0.5) / pr + 0.5;
    c->cp.pr_on = pr != 1.0;
    c->cp.cpr = c->cp.pr_on ? 1.0 / p->tau - 1.0 / tau_pr : 0.0;
    c->cp.cprf = (float)c->cp.cpr;
  }
  c->store = p->prec == SLLBM_PREC_F32 ? kStoreF32 : (p->prec == SLLBM_PREC_BF16_STORE ? kStoreBF16 : kStoreF64);
  c->elem = c->store == kStoreF32 ? 4 : (c->store == kStoreBF16 ? 2 : 8);
  // Plane layout: ghost cells around the interior (8 columns left, 4 rows above, enough right
  // and below for the last tile's halo), rows 16-byte aligned for every storage type.  Mapped
  // grids get 16 on every side: their staged windows follow the departure displacement, which
  // may reach a few vertex spacings across a periodic seam.
  if (g->map != SLLBM_MAP_IDENTITY) {
    c->gx = 16;
    c->gy = 16;
    c->gyb = 24;
  }
  c->gxr = (c->nx + 31) / 32 * 32 - c->nx + c->gx;
  c->rows_alloc = c->gy + c->ny + c->gyb;
  c->pitchv = (c->gx + c->nx + c->gxr + 7) / 8 * 8;
  c->xs = (c->store == kStoreF64 || c->nq1 == 3) ? 1 : 2;
  c->pitch = c->pitchv * c->xs;
  c->plane_stride = (size_t)c->rows_alloc * c->pitch;
  c->ps = (c->xs == 2) ? 1 : (ptrdiff_t)c->nq * c->plane_stride;
  c->ghost.on = 0;
  c->ghost.px = c->ax.periodic;
  c->ghost.py = c->ay.periodic;
  c->ghost.nx = c->nx;
  c->ghost.ny = c->ny;
  c->ghost.xlo = -c->gx;
  c->ghost.xhi = c->nx + c->gxr;
  c->ghost.ylo = -c->gy;
  c->ghost.yhi = c->ny + c->gyb;
  sllbm_status s;
  const size_t state_elems = (size_t)2 * c->nq * c->rows_alloc * c->pitchv;
  for (int k = 0; k < 2; ++k) {
    void* ptr = nullptr;
    s = dalloc(c, reinterpret_cast<char**>(&ptr), state_elems * c->elem);
    if (s != SLLBM_OK) { sllbm_destroy(c); return s; }
    c->alloc[k] = ptr;
    c->state[k] = static_cast<char*>(ptr) + ((size_t)c->gy * c->pitch + (size_t)c->gx * c->xs) * c->elem;
    if (cudaMemsetAsync(ptr, 0, state_elems * c->elem, c->stream) != cudaSuccess) {
      sllbm_destroy(c);
      return SLLBM_ERR_CUDA;
    }
  }
  const int nblocks = moments_blocks(c->nv);
  if ((s = dalloc(c, &c->A, c->nv)) != SLLBM_OK || (s = dalloc(c, &c->partials, 2 * (size_t)nblocks)) != SLLBM_OK ||
      (s = dalloc(c, &c->sums, 2)) != SLLBM_OK || (s = dalloc(c, &c->flag, 1)) != SLLBM_OK) {
    sllbm_destroy(c);
    return s;
  }
  if (cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream) != cudaSuccess) {
    sllbm_destroy(c);
    return SLLBM_ERR_CUDA;
  }
  *out = c;
  return SLLBM_OK;
}

sllbm_status sllbm_set_stream(sllbm_ctx* c, void* stream) {
  if (!c) return SLLBM_ERR_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  c->graph_off = false;   // the step graph (if built) launches on any stream; try capture again
  return SLLBM_OK;
}

sllbm_status sllbm_grid_info(const sllbm_ctx* c, int* nx, int* ny, int* npop) {
  if (!c) return SLLBM_ERR_ARG;
  if (nx) *nx = c->nx;
  if (ny) *ny = c->ny;
  if (npop) *npop = c->npop;
  return SLLBM_OK;
}

sllbm_status sllbm_state_bytes(const sllbm_ctx* c, size_t* bytes) {
  if (!c || !bytes) return SLLBM_ERR_ARG;
  *bytes = (size_t)c->npop * c->nq * c->nv * c->elem;
  return SLLBM_OK;
}

sllbm_status sllbm_vertex_coords(sllbm_ctx* c, double* x, double* y) {
  if (!c || !x || !y) return fail(c, SLLBM_ERR_ARG, "null pointer");
  CUDA_TRY(c, launch_vertex_coords(geom_args(c), x, y, c->stream));
  return SLLBM_OK;
}

sllbm_status sllbm_vertex_weights(sllbm_ctx* c, double* A) {
  if (!c || !A) return fail(c, SLLBM_ERR_ARG, "null pointer");
  if (!c->precomputed) return fail(c, SLLBM_ERR_STATE, "precompute_departures first");
  CUDA_TRY(c, cudaMemcpyAsync(A, c->A, sizeof(double) * c->nv, cudaMemcpyDeviceToDevice, c->stream));
  return SLLBM_OK;
}

sllbm_status sllbm_precompute_departures(sllbm_ctx* c) {
  if (!c) return SLLBM_ERR_ARG;
  GeomArgs g = geom_args(c);
  const bool mapped = c->map.kind != SLLBM_MAP_IDENTITY;
  if (!mapped) {  // per-axis tables
    if (!c->offx) {
      TRY(dalloc(c, &c->offx, kQ1 * (size_t)c->nx));
      TRY(dalloc(c, &c->offy, kQ1 * (size_t)c->ny));
      TRY(dalloc(c, &c->wx, kQ1 * (size_t)c->nx * (c->P + 1)));
      TRY(dalloc(c, &c->wy, kQ1 * (size_t)c->ny * (c->P + 1)));
      TRY(dalloc(c, &c->wx64, kQ1 * (size_t)c->nx * (c->P + 1)));
      TRY(dalloc(c, &c->wy64, kQ1 * (size_t)c->ny * (c->P + 1)));
    }
    CUDA_TRY(c, launch_axis_tables(c->ax, c->cs, c->p.dt, c->offx, c->wx, c->wx64, c->stream));
    CUDA_TRY(c, launch_axis_tables(c->ay, c->cs, c->p.dt, c->offy, c->wy, c->wy64, c->stream));
    std::vector<int> ox(c->nq1 * (size_t)c->nx), oy(c->nq1 * (size_t)c->ny);
    CUDA_TRY(c, cudaMemcpyAsync(ox.data(), c->offx, ox.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(oy.data(), c->offy, oy.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->offx_lo = *std::min_element(ox.begin(), ox.end());
    c->offx_hi = *std::max_element(ox.begin(), ox.end()) + c->P;
    c->offy_lo = *std::min_element(oy.begin(), oy.end());
    c->offy_hi = *std::max_element(oy.begin(), oy.end()) + c->P;
  }
  c->n_fix = 0;
  if (c->nq1 == 3) {
    c->kernel = kKernelQ9;
  } else if (c->store == kStoreF64) {
    c->kernel = kKernelPlainF64;
  } else if (!mapped) {
    TRY(build_uniform_pattern(c));
    c->kernel = c->ut.valid ? kKernelUniform : kKernelGather;
  } else {
    c->kernel = kKernelGather;
  }
  const bool need_desc = mapped || (c->kernel == kKernelGather);
  if (need_desc) {
    if (!c->dcx) {
      const size_t n = (size_t)kQ * c->nv;
      TRY(dalloc(c, &c->dcx, n));
      TRY(dalloc(c, &c->dcy, n));
      TRY(dalloc(c, &c->dr, n));
      TRY(dalloc(c, &c->ds, n));
      TRY(dalloc(c, &c->dr64, n));
      TRY(dalloc(c, &c->ds64, n));
    }
    CUDA_TRY(c, launch_descriptors(g, c->dcx, c->dcy, c->dr, c->ds, c->dr64, c->ds64, c->stream));
  }
  if (mapped && c->store != kStoreF64 && c->kernel != kKernelQ9) {
    TRY(build_mapped_tiles(c));
    if (c->mt.valid) c->kernel = kKernelMapped;
  }
  c->q9_tma = 0;
  if (c->kernel == kKernelQ9 && (c->store == kStoreF32 || c->store == kStoreBF16) && !mapped) {
    StepArgs a = step_args(c, c->state[0], c->state[1]);
    a.mapped = 0;
    c->q9_tma = q9_tma_usable(a, c->elem) ? 1 : 0;
  }
  c->ghost.on = (c->kernel == kKernelUniform || c->kernel == kKernelMapped || c->q9_tma) &&
                (c->ax.periodic || c->ay.periodic);
  double glx[8], glw[8];
  const int ngl = c->P + 3;
  gauss_legendre01(ngl, glx, glw);
  CUDA_TRY(c, launch_vertex_weights(g, glx, glw, ngl, c->A, c->stream));
  int flag = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (flag & 2) return fail(c, SLLBM_ERR_NEWTON, "Newton inversion of the grid map did not converge");
  c->precomputed = true;
  c->transposed = false;
  return SLLBM_OK;
}

sllbm_status sllbm_init_equilibrium(sllbm_ctx* c, const double* rho, const double* u, const double* v,
                                    const double* T) {
  if (!c || !rho || !u || !v || !T) return fail(c, SLLBM_ERR_ARG, "null pointer");
  if (!c->precomputed) return fail(c, SLLBM_ERR_STATE, "precompute_departures first");
  InitArgs a{};
  a.rho = rho;
  a.u = u;
  a.v = v;
  a.T = T;
  a.dst = c->state[c->cur];
  a.nx = c->nx;
  a.ny = c->ny;
  a.pitch = c->pitch;
  a.nv = c->nv;
  a.plane_stride = c->plane_stride;
  a.xs = c->xs;
  a.ps = c->ps;
  a.cs = c->cs;
  a.cp = c->cp;
  a.store = c->store;
  CUDA_TRY(c, launch_init_equilibrium(a, c->stream));
  CUDA_TRY(c, fill_ghosts(c));
  c->initialized = true;
  return SLLBM_OK;
}

// The side stream and its two events of the fix-up gather (created on first use).
static cudaError_t ensure_side(sllbm_ctx* c) {
  if (c->side) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&c->side_ev[k], cudaEventDisableTiming);
  return e;
}

static cudaError_t enqueue_step(sllbm_ctx* c, float* mom = nullptr) {
  StepArgs a = step_args(c, c->state[c->cur], c->state[c->cur ^ 1]);
  a.mom = mom;
  cudaError_t e;
  switch (c->kernel) {
    case kKernelUniform:
      if (c->n_fix > 0) {
        // vertices off the cell-periodic pattern: the gather kernel reads the same source and
        // writes other vertices than the fused kernel, so it runs on a side stream beside it
        // (filling the SMs the persistent kernel's tail leaves idle); the step ends when both do
        if ((e = ensure_side(c)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->side_ev[0], c->stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(c->side, c->side_ev[0], 0)) != cudaSuccess) return e;
        e = launch_step_uniform(a, c->ut, c->store, c->stream);
        if (e != cudaSuccess) return e;
        StepArgs f = a;
        f.vlist = c->fix_list;
        f.nlist = c->n_fix;
        f.mapped = 0;
        if ((e = launch_step_gather(f, c->store, c->side)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->side_ev[1], c->side)) != cudaSuccess) return e;
        e = cudaStreamWaitEvent(c->stream, c->side_ev[1], 0);
      } else {
        e = launch_step_uniform(a, c->ut, c->store, c->stream);
      }
      break;
    case kKernelMapped:
      e = launch_step_mapped(a, c->mt, c->store, c->stream);
      if (e == cudaSuccess && c->n_fix > 0) {  // tiles whose windows did not fit
        a.vlist = c->fix_list;
        a.nlist = c->n_fix;
        a.mapped = 1;
        e = launch_step_gather(a, c->store, c->stream);
      }
      break;
    case kKernelPlainF64: e = launch_step_plain_f64(a, c->stream); break;
    case kKernelQ9: e = launch_step_q9(a, c->store, c->stream); break;
    default: e = launch_step_gather(a, c->store, c->stream); break;
  }
  if (e == cudaSuccess) c->cur ^= 1;
  return e;
}

// A CUDA graph of two steps, from state buffer 0 through 1 back to 0: every launch of the steps
// (the fused kernel, the fix-up gather on its side stream and the events between them) with its
// parameters as the step's host set-up computed them.  The buffers and tables it refers to live
// as long as the context, so the graph stays valid.
static cudaError_t build_step_graph(sllbm_ctx* c) {
  cudaError_t e = ensure_side(c);   // nothing is created while capturing
  if (e != cudaSuccess) return e;
  if (c->stream == nullptr || c->stream == cudaStreamLegacy ||
      cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();   // the legacy default stream (or another one capture refuses): no graph
    c->graph_off = true;
    return cudaSuccess;
  }
  const int cur0 = c->cur;
  cudaError_t e1 = enqueue_step(c);
  if (e1 == cudaSuccess) e1 = enqueue_step(c);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->stream, &g);
  c->cur = cur0;   // the captured steps did not run
  if (e1 != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e1 != cudaSuccess ? e1 : e;
  }
  e = cudaGraphInstantiate(&c->step_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) c->step_graph = nullptr;
  return e;
}

sllbm_status sllbm_step(sllbm_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return fail(c, SLLBM_ERR_ARG, "bad arguments");
  if (!c->precomputed || !c->initialized) return fail(c, SLLBM_ERR_STATE, "precompute and init first");
  int k = 0;
  if (nsteps >= kGraphMinSteps && !c->graph_off && dense_bytes(c) <= kGraphMaxStateBytes) {
    // pairs of steps replay the two-step graph: one launch on the stream in place of each step's
    // launches, event records and host set-up (small grids are bound by those)
    if (c->cur != 0) {
      CUDA_TRY(c, enqueue_step(c));
      ++k;
    }
    if (!c->step_graph) CUDA_TRY(c, build_step_graph(c));
    if (c->step_graph)
      for (; k + 2 <= nsteps; k += 2) CUDA_TRY(c, cudaGraphLaunch(c->step_graph, c->stream));
  }
  for (; k < nsteps; ++k) CUDA_TRY(c, enqueue_step(c));
  return SLLBM_OK;
}

sllbm_status sllbm_step_moments(sllbm_ctx* c, float* moments) {
  if (!c || !moments) return fail(c, SLLBM_ERR_ARG, "null pointer");
  if (c->nq1 != kQ1) return fail(c, SLLBM_ERR_UNSUPPORTED, "the moments epilogue covers the D2Q25 set");
  if (!c->precomputed || !c->initialized) return fail(c, SLLBM_ERR_STATE, "precompute and init first");
  CUDA_TRY(c, enqueue_step(c, moments));
  return SLLBM_OK;
}

const char* sllbm_step_kernel_name(const sllbm_ctx* c) {
  if (!c) return "none";
  switch (c->kernel) {
    case kKernelUniform: return "uniform_fused";
    case kKernelPlainF64: return "plain_f64";
    case kKernelMapped: return "mapped_fused";
    case kKernelQ9: return "d2q9";
    default: return "gather";
  }
}

int sllbm_launches_per_step(const sllbm_ctx* c) {
  if (!c) return 0;
  return ((c->kernel == kKernelUniform || c->kernel == kKernelMapped) && c->n_fix > 0) ? 2 : 1;
}


sllbm_status sllbm_get_state(sllbm_ctx* c, void* dst) {
  if (!c || !dst) return fail(c, SLLBM_ERR_ARG, "null pointer");
  TRY(copy_state(c, dst, c->state[c->cur], false, cudaMemcpyDeviceToDevice));
  return SLLBM_OK;
}

sllbm_status sllbm_set_state(sllbm_ctx* c, const void* src) {
  if (!c || !src) return fail(c, SLLBM_ERR_ARG, "null pointer");
  TRY(copy_state(c, c->state[c->cur], src, true, cudaMemcpyDeviceToDevice));
  CUDA_TRY(c, fill_ghosts(c));
  c->initialized = true;
  return SLLBM_OK;
}

sllbm_status sllbm_step_host(sllbm_ctx* c, const void* in, void* out, int nsteps) {
  if (!c || !in || !out || nsteps < 0) return fail(c, SLLBM_ERR_ARG, "bad arguments");
  if (!c->precomputed) return fail(c, SLLBM_ERR_STATE, "precompute_departures first");
  TRY(copy_state(c, c->state[c->cur], in, true, cudaMemcpyHostToDevice));
  CUDA_TRY(c, fill_ghosts(c));
  c->initialized = true;
  for (int k = 0; k < nsteps; ++k) CUDA_TRY(c, enqueue_step(c));
  TRY(copy_state(c, out, c->state[c->cur], false, cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return SLLBM_OK;
}

sllbm_status sllbm_moments(sllbm_ctx* c, float* rho, float* u, float* v, float* T, double* me) {
  if (!c) return SLLBM_ERR_ARG;
  if (!c->initialized) return fail(c, SLLBM_ERR_STATE, "no state");
  MomentArgs a{};
  a.src = c->state[c->cur];
  a.nx = c->nx;
  a.ny = c->ny;
  a.pitch = c->pitch;
  a.nv = c->nv;
  a.plane_stride = c->plane_stride;
  a.xs = c->xs;
  a.ps = c->ps;
  a.cs = c->cs;
  a.cp = c->cp;
  a.store = c->store;
  a.A = c->precomputed ? c->A : nullptr;
  a.rho = rho;
  a.u = u;
  a.v = v;
  a.T = T;
  a.partials = me ? c->partials : nullptr;
  a.sums = c->sums;
  a.flag = c->flag;
  CUDA_TRY(c, launch_moments(a, c->stream));
  int flag = 0;
  if (me) CUDA_TRY(c, cudaMemcpyAsync(me, c->sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (flag & 4) return fail(c, SLLBM_ERR_CUDA, "a staging copy of the fused kernel timed out");
  if (flag & 1) return fail(c, SLLBM_ERR_UNSTABLE, "non-positive or non-finite density/temperature");
  return SLLBM_OK;
}

// ---- transposed stencils for the adjoint (host build from the FP64 tables) ----
// Per axis, component and node j: the (vertex, weight) pairs of the vertices whose stencil reads
// j, in ascending vertex order (deterministic).
struct AxisTranspose {
  std::vector<std::vector<std::pair<int, float>>> rows;   // [comp * n + j]
  size_t max_deg = 0;
  int max_offset = 0;   // largest |vertex - node| over all entries (the short way round if periodic)
};

static sllbm_status axis_transpose(sllbm_ctx* c, const AxisK& ax, const int* off_dev, const double* w_dev,
                                   AxisTranspose* t) {
  const int n = ax.nv, P = c->P;
  std::vector<int> off((size_t)kQ1 * n);
  std::vector<double> w((size_t)kQ1 * n * (P + 1));
  CUDA_TRY(c, cudaMemcpyAsync(off.data(), off_dev, off.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(w.data(), w_dev, w.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  t->rows.assign((size_t)kQ1 * n, {});
  for (int comp = 0; comp < kQ1; ++comp)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k <= P; ++k) {
        const int src = wrap_index(j + off[(size_t)comp * n + j] + k, n, ax.periodic);
        t->rows[(size_t)comp * n + src].push_back({j, (float)w[((size_t)comp * n + j) * (P + 1) + k]});
      }
  for (const auto& r : t->rows) t->max_deg = std::max(t->max_deg, r.size());
  for (size_t r = 0; r < t->rows.size(); ++r)
    for (const auto& e : t->rows[r]) {
      int d = e.first - (int)(r % n);
      if (ax.periodic) {
        if (d > n / 2) d -= n;
        if (d < -n / 2) d += n;
      }
      t->max_offset = std::max(t->max_offset, d < 0 ? -d : d);
    }
  return SLLBM_OK;
}

// Fixed-width copy of a transpose: kw entries per (comp, node), padded with weight 0 on the node.
static sllbm_status upload_transpose(sllbm_ctx* c, const AxisTranspose& t, int n, int kw, int** col_dev,
                                     float** w_dev, int** deg_dev) {
  std::vector<int> col(t.rows.size() * kw), deg(t.rows.size());
  std::vector<float> wt(t.rows.size() * kw, 0.f);
  for (size_t r = 0; r < t.rows.size(); ++r) {
    deg[r] = (int)t.rows[r].size();
    for (int k = 0; k < kw; ++k) {
      const bool have = (size_t)k < t.rows[r].size();
      col[r * kw + k] = have ? t.rows[r][k].first : (int)(r % n);
      wt[r * kw + k] = have ? t.rows[r][k].second : 0.f;
    }
  }
  TRY(dalloc(c, col_dev, col.size()));
  TRY(dalloc(c, w_dev, wt.size()));
  TRY(dalloc(c, deg_dev, deg.size()));
  CUDA_TRY(c, cudaMemcpy(*col_dev, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(*w_dev, wt.data(), wt.size() * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(*deg_dev, deg.data(), deg.size() * sizeof(int), cudaMemcpyHostToDevice));
  return SLLBM_OK;
}

// Dense copy of a transpose for the one-pass S^T: per (comp, node j), dw weights indexed by the
// source offset d + h, d = source - j in [-h, h] (the short way round a periodic axis), 0 where
// no entry has that offset.
static sllbm_status upload_dense_transpose(sllbm_ctx* c, const AxisTranspose& t, int n, bool periodic, int h,
                                           int dw, float** dense_dev) {
  std::vector<float> dense(t.rows.size() * dw, 0.f);
  for (size_t r = 0; r < t.rows.size(); ++r)
    for (const auto& e : t.rows[r]) {
      int d = e.first - (int)(r % n);
      if (periodic) {
        if (d > n / 2) d -= n;
        if (d < -n / 2) d += n;
      }
      if (d < -h || d > h) return fail(c, SLLBM_ERR_UNSUPPORTED, "adjoint: stencil offset beyond the halo");
      dense[r * dw + (d + h)] += e.second;
    }
  TRY(dalloc(c, dense_dev, dense.size()));
  CUDA_TRY(c, cudaMemcpy(*dense_dev, dense.data(), dense.size() * sizeof(float), cudaMemcpyHostToDevice));
  return SLLBM_OK;
}

static double lagrange_host(const double* nodes, int P, int a, double r) {
  double acc = 1.0;
  for (int b = 0; b <= P; ++b)
    if (b != a) acc *= (r - nodes[b]) / (nodes[a] - nodes[b]);
  return acc;
}

static sllbm_status build_mapped_transpose(sllbm_ctx* c) {
  const long long nv = c->nv;
  const int P = c->P, nx = c->nx, ny = c->ny;
  const size_t n = (size_t)kQ * nv;
  std::vector<int> cx(n), cy(n);
  std::vector<double> r(n), s(n);
  CUDA_TRY(c, cudaMemcpyAsync(cx.data(), c->dcx, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(cy.data(), c->dcy, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(r.data(), c->dr64, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(s.data(), c->ds64, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const int per = (P + 1) * (P + 1);
  std::vector<long long> ptr((size_t)kQ * (nv + 1), 0);
  for (int i = 0; i < kQ; ++i) {
    long long* p0 = &ptr[(size_t)i * (nv + 1)];
    for (long long v = 0; v < nv; ++v) {
      const size_t d = (size_t)i * nv + v;
      for (int kb = 0; kb <= P; ++kb)
        for (int ka = 0; ka <= P; ++ka) {
          const int sx = wrap_index(cx[d] * P + ka, nx, c->ax.periodic);
          const int sy = wrap_index(cy[d] * P + kb, ny, c->ay.periodic);
          p0[(long long)sy * nx + sx + 1]++;
        }
    }
  }
  long long total = 0;
  for (int i = 0; i < kQ; ++i) {
    long long* p0 = &ptr[(size_t)i * (nv + 1)];
    p0[0] = total;
    for (long long v = 0; v < nv; ++v) p0[v + 1] += p0[v];
    total = p0[nv];
  }
  (void)per;
  std::vector<int> col(total);
  std::vector<float> wt(total);
  std::vector<long long> fill(ptr.begin(), ptr.end());
  for (int i = 0; i < kQ; ++i)
    for (long long v = 0; v < nv; ++v) {
      const size_t d = (size_t)i * nv + v;
      for (int kb = 0; kb <= P; ++kb)
        for (int ka = 0; ka <= P; ++ka) {
          const int sx = wrap_index(cx[d] * P + ka, nx, c->ax.periodic);
          const int sy = wrap_index(cy[d] * P + kb, ny, c->ay.periodic);
          const long long e = fill[(size_t)i * (nv + 1) + (long long)sy * nx + sx]++;
          col[e] = (int)v;
          wt[e] = (float)(lagrange_host(c->ax.nodes, P, ka, r[d]) * lagrange_host(c->ay.nodes, P, kb, s[d]));
        }
    }
  TRY(dalloc(c, &c->tm_ptr, ptr.size()));
  TRY(dalloc(c, &c->tm_col, (size_t)total));
  TRY(dalloc(c, &c->tm_w, (size_t)total));
  CUDA_TRY(c, cudaMemcpy(c->tm_ptr, ptr.data(), ptr.size() * sizeof(long long), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->tm_col, col.data(), (size_t)total * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpy(c->tm_w, wt.data(), (size_t)total * sizeof(float), cudaMemcpyHostToDevice));
  return SLLBM_OK;
}

sllbm_status sllbm_adjoint_step(sllbm_ctx* c, const float* lam_in, float* lam_out, const float* moments) {
  if (!c || !lam_in || !lam_out || !moments) return fail(c, SLLBM_ERR_ARG, "null pointer");
  if (lam_in == lam_out) return fail(c, SLLBM_ERR_ARG, "lambda_in and lambda_out alias");
  if (c->cp.pr_on || c->cp.iso)
    return fail(c, SLLBM_ERR_UNSUPPORTED, "the adjoint covers the thermal BGK collision (Pr = 1) only");
  if (!c->precomputed) return fail(c, SLLBM_ERR_STATE, "precompute_departures first");
  const bool mapped = c->map.kind != SLLBM_MAP_IDENTITY;
  if (!c->transposed) {
    if (mapped) {
      TRY(dalloc(c, &c->mu, (size_t)2 * kQ * c->nv));
      TRY(build_mapped_transpose(c));
    } else {
      AxisTranspose tx, ty;
      TRY(axis_transpose(c, c->ax, c->offx, c->wx64, &tx));
      TRY(axis_transpose(c, c->ay, c->offy, c->wy64, &ty));
      const int kw = (int)((std::max(tx.max_deg, ty.max_deg) + 3) / 4 * 4);   // 16-byte rows
      if (kw > 16) return fail(c, SLLBM_ERR_UNSUPPORTED, "adjoint: more than 16 stencils read one node");
      TRY(upload_transpose(c, tx, c->nx, kw, &c->tx_col, &c->tx_w, &c->tx_deg));
      TRY(upload_transpose(c, ty, c->ny, kw, &c->ty_col, &c->ty_w, &c->ty_deg));
      c->tkw = kw;
      c->thalo = std::max(tx.max_offset, ty.max_offset);
      if (adjoint_tma_usable(c->nx, c->ny, c->ax.periodic, c->ay.periodic, c->thalo)) {
        // ghost-padded pairs for the one-pass S^T; rows of a multiple of 4 pairs (32 bytes)
        c->mu_g = kAdjGhost;
        c->mu_pitch = (c->nx + 2 * kAdjGhost + 3) / 4 * 4;
        c->mu_rows = c->ny + 2 * kAdjGhost;
        const size_t n = (size_t)2 * kQ * c->mu_rows * c->mu_pitch;
        TRY(dalloc(c, &c->mu, n));
        CUDA_TRY(c, cudaMemsetAsync(c->mu, 0, n * sizeof(float), c->stream));   // ghosts never written
        c->thalo_k = adjoint_tma_halo(c->thalo);
        c->tdw = adjoint_dense_width(c->thalo_k);
        TRY(upload_dense_transpose(c, tx, c->nx, c->ax.periodic, c->thalo_k, c->tdw, &c->tx_dense));
        TRY(upload_dense_transpose(c, ty, c->ny, c->ay.periodic, c->thalo_k, c->tdw, &c->ty_dense));
      } else {
        TRY(dalloc(c, &c->mu, (size_t)2 * kQ * c->nv));
        TRY(dalloc(c, &c->atmp, (size_t)kQ * c->nv));
      }
    }
    c->transposed = true;
  }
  AdjointArgs a{};
  a.lam_in = lam_in;
  a.lam_out = lam_out;
  a.mu = reinterpret_cast<float2*>(c->mu);
  a.mu_g = c->mu_g;
  a.mu_pitch = c->mu_g > 0 ? c->mu_pitch : c->nx;
  a.mu_rows = c->mu_g > 0 ? c->mu_rows : c->ny;
  a.flag = c->flag;
  a.moments = moments;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nv = c->nv;
  a.cs = c->cs;
  a.cp = c->cp;
  a.mapped = mapped;
  a.kw = c->tkw;
  a.tx_col = c->tx_col;
  a.tx_w = c->tx_w;
  a.tx_deg = c->tx_deg;
  a.ty_col = c->ty_col;
  a.ty_w = c->ty_w;
  a.ty_deg = c->ty_deg;
  a.tmp = c->atmp;
  a.periodic_x = c->ax.periodic;
  a.periodic_y = c->ay.periodic;
  a.halo = c->thalo;
  a.tx_dense = c->tx_dense;
  a.ty_dense = c->ty_dense;
  a.dhalo = c->thalo_k;
  a.dw = c->tdw;
  a.tm_ptr = c->tm_ptr;
  a.tm_col = c->tm_col;
  a.tm_w = c->tm_w;
  CUDA_TRY(c, launch_adjoint_step(a, c->stream));
  return SLLBM_OK;
}

sllbm_status sllbm_init_equilibrium_vjp(sllbm_ctx* c, const double* rho, const double* u, const double* v,
                                        const double* T, const float* lam0, float* du, float* dv) {
  if (!c || !rho || !u || !v || !T || !lam0 || !du || !dv) return fail(c, SLLBM_ERR_ARG, "null pointer");
  if (c->nq1 != kQ1) return fail(c, SLLBM_ERR_UNSUPPORTED, "the equilibrium VJP covers the D2Q25 set");
  InitVjpArgs a{};
  a.rho = rho;
  a.u = u;
  a.v = v;
  a.T = T;
  a.lam = lam0;
  a.du = du;
  a.dv = dv;
  a.nv = c->nv;
  a.cs = c->cs;
  a.cp = c->cp;
  CUDA_TRY(c, launch_init_vjp(a, c->stream));
  return SLLBM_OK;
}

}  // extern "C"
