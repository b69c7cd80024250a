// Host-side launch interface of the SLLBM kernels (one translation unit per kernel family).
#pragma once

#include <stddef.h>

#include "sllbm_internal.cuh"

namespace sllbm {

enum StoreKind { kStoreF32 = 0, kStoreBF16 = 1, kStoreF64 = 2 };

// Everything a step kernel needs.  Uniform grids use the per-axis tables (off*, w*), transformed
// grids (or uniform grids with departure offsets beyond the fused kernel's halo) the per-(velocity,
// vertex) descriptors (dc*, dr/ds).  Offsets off[c][j] are stencil start minus vertex index.
struct StepArgs {
  const void* src;
  void* dst;
  int nx, ny, pitch, periodic_x, periodic_y, P;
  long long nv;
  // State layout: value (pop, i, y, x) at src[i * plane_stride + pop * ps + y * pitch + x * xs]
  // (interior origin).  FP32/BF16 storage interleaves f and g (xs = 2, ps = 1); FP64 is planar.
  size_t plane_stride;  // elements between velocity planes
  int xs;               // elements between neighbouring vertices of a row
  ptrdiff_t ps;         // elements between the f and g values of one (velocity, vertex)
  const int* offx;
  const int* offy;
  const float* wx;      // [5][nx][P+1]
  const float* wy;      // [5][ny][P+1]
  const double* wx64;
  const double* wy64;
  const int* dcx;       // [25][nv] departure cell index in x
  const int* dcy;
  const float* dr;      // [25][nv] local reference coordinate in the cell
  const float* ds;
  const double* dr64;
  const double* ds64;
  float nodesf[5];
  double nodes[5];
  Consts cs;
  CollideK cp;
  int* flag;            // bit 0: unstable
  int mapped;           // 1: use descriptors
  // fused uniform kernel geometry
  int offx_min, offx_max, offy_min, offy_max;
  // optional vertex list (gather kernel only): process vlist[0..nlist) instead of every vertex
  const int* vlist;
  long long nlist;
  GhostK ghost;         // periodic images to keep up to date in the ghost cells
  // optional: (rho, u, v, theta) of each vertex's collision, dense [4][ny][nx] FP32 (plane
  // stride nv); null to skip
  float* mom;
  // D2Q9, FP32 or BF16 storage on a uniform grid: the TMA-staged kernel (the ghost cells hold
  // the periodic images, kept by its writes); gx, gy, rows_alloc as in UniformTables
  int q9_tma;
  int gx, gy, rows_alloc;
};

// Cell-periodic pattern of a uniform grid (see step_uniform.cu): per velocity component and
// local node, the y interpolation as a band of 2p+1 taps around the vertex and the x taps.
struct UniformTables {
  bool valid;
  double wy_pat[kQ1][4][5];   // [b][l][alpha]
  double wx_pat[kQ1][4][5];   // [a][k][alpha]
  int dy_pat[kQ1][4];         // [b][l]: stencil start - vertex row, in [-p, 0]
  int dx_pat[kQ1][4];         // [a][k]: stencil start - vertex column, in [-p, 0]
  const unsigned char* std_x; // [nx]: column follows the pattern
  const unsigned char* std_y; // [ny]
  int gx, gy, rows_alloc;     // ghost columns/rows before the interior origin; rows per plane
};

// Fused shared-memory step for mapped grids: per (tile of kMappedTileX x kMappedTileY vertices,
// velocity plane) one staged window of the source plane; writes only vertices of tiles marked in
// tile_ok.  cudaErrorNotSupported if the tables are not valid.
constexpr int kMappedTileX = 32, kMappedTileY = 8;
struct MappedTables {
  bool valid;
  // departure records, [3][25][rows][dpitch] 32-bit words (rows = ny rounded up to the tile):
  // (ly << 16) | lx, the stencil origin inside the window; r and s, the local coordinates
  const uint32_t* rec;
  int dpitch;
  const int2* org;            // [ntiles][25]: window origin (node column, node row)
  const unsigned char* tile_ok;
  int bw, bh;                 // window: bw vertices x bh rows
  int gx, gy, rows_alloc;     // ghost columns/rows before the interior origin; rows per plane
  float wc[4][5];             // W_alpha(t) = sum_j wc[alpha-1][j] t^j, t = r - 1/2
};
cudaError_t launch_step_mapped(const StepArgs& a, const MappedTables& t, int store, cudaStream_t s);
size_t mapped_smem_bytes(int bw, int bh, int store);

// Generic FP32 gather step (one thread per vertex, (p+1)^2 gathers per plane from L1/L2).
cudaError_t launch_step_gather(const StepArgs& a, int store, cudaStream_t s);
// Fused shared-memory step for uniform grids (pattern band interpolation); writes only the
// vertices marked in std_x/std_y.  cudaErrorNotSupported if the tables are not valid.
cudaError_t launch_step_uniform(const StepArgs& a, const UniformTables& t, int store, cudaStream_t s);
// Plain FP64 step on full populations.
cudaError_t launch_step_plain_f64(const StepArgs& a, cudaStream_t s);
// D2Q9 step (isothermal, one population, planar storage): FP32 arithmetic on FP32/BF16
// deviations or FP64 on full populations; per-axis tables or, with a.mapped, descriptors.
cudaError_t launch_step_q9(const StepArgs& a, int store, cudaStream_t s);
// Whether the TMA-staged D2Q9 kernel can take this uniform grid with elem-byte storage (FP32 or
// BF16: its window fits the shared memory and the ghost cells); the host then keeps the periodic
// images in the ghost cells.
bool q9_tma_usable(const StepArgs& a, int elem);

// ---- precompute (FP64) ----
struct GeomArgs {
  AxisK ax, ay;
  MapK map;
  Consts cs;
  double dt;
  int nx, ny;
  long long nv;
  int* flag;            // bit 1: Newton failure
};
cudaError_t launch_axis_tables(const AxisK& ax, const Consts& cs, double dt, int* off, float* w32,
                               double* w64, cudaStream_t s);
cudaError_t launch_descriptors(const GeomArgs& g, int* dcx, int* dcy, float* dr, float* ds,
                               double* dr64, double* ds64, cudaStream_t s);
cudaError_t launch_vertex_coords(const GeomArgs& g, double* x, double* y, cudaStream_t s);
cudaError_t launch_vertex_weights(const GeomArgs& g, const double* gl_x, const double* gl_w,
                                  int ngl, double* A, cudaStream_t s);
struct InitArgs {
  const double *rho, *u, *v, *T;
  void* dst;
  int nx, ny, pitch;
  long long nv;
  size_t plane_stride;
  int xs;
  ptrdiff_t ps;
  Consts cs;
  CollideK cp;
  int store;
};
cudaError_t launch_init_equilibrium(const InitArgs& a, cudaStream_t s);
// Dense [npop][nq][ny][nx] <-> internal layout (interior origin `internal`), element size `elem`,
// for the dense planes [plane0, plane0 + nplanes) (plane = pop * nq + velocity).
cudaError_t launch_state_convert(const void* src, void* dst, bool to_internal, int elem, int plane0,
                                 int nplanes, int nq, int nx, int ny, int pitch, size_t plane_stride,
                                 int xs, ptrdiff_t ps, cudaStream_t s);
// Dense [npop][nq][ny][nx] <-> interleaved (f, g) pairs (xs = 2, ps = 1) for the velocity planes
// [i0, i0 + ni), both populations at once (elem 4: FP32, 2: BF16).
cudaError_t launch_pair_convert(const void* src, void* dst, bool to_internal, int elem, int i0, int ni, int npop,
                                int nq, int nx, int ny, int pitch, size_t plane_stride, cudaStream_t s);
// Copy the periodic images of interior vertices into the ghost cells of `planes` planes (clamped
// copies on non-periodic axes).  `origin`: interior origin of plane 0; elem: bytes per element.
cudaError_t launch_ghost_fill(void* origin, int elem, size_t plane_stride, int pitch, int planes,
                              const GhostK& g, cudaStream_t s);

// ---- moments and reductions ----
struct MomentArgs {
  const void* src;
  int nx, ny, pitch;
  long long nv;
  size_t plane_stride;
  int xs;
  ptrdiff_t ps;
  Consts cs;
  CollideK cp;
  int store;
  const double* A;
  float *rho, *u, *v, *T;
  double* partials;   // [2][nblocks] scratch for the deterministic reduction
  double* sums;       // [2] device result (may be null when partials is null)
  int* flag;
};
int moments_blocks(long long nv);
cudaError_t launch_moments(const MomentArgs& a, cudaStream_t s);

// ---- adjoint ----
struct AdjointArgs {
  const float* lam_in;
  float* lam_out;
  // scratch: J_C^T lambda as (f, g) pairs, [25][mu_rows][mu_pitch] with mu_g ghost columns and
  // rows before the interior origin: dense (mu_g = 0, pitch nx, ny rows) for the two-pass and
  // mapped S^T, ghost-padded (mu_g = kAdjGhost, periodic images kept by J_C^T) for the one-pass S^T
  float2* mu;
  int mu_pitch, mu_rows, mu_g;
  int* flag;           // bit 2: a staging copy of the one-pass S^T timed out
  const float* moments;  // [4][nv]
  int nx, ny;
  long long nv;
  Consts cs;
  CollideK cp;
  // transposed stencils: uniform per axis (fixed width kw per (component, node), padded with
  // zero weights), mapped per velocity (CSR over vertex index)
  int mapped;
  int kw;
  const int* tx_col;   // [5][nx][kw]
  const float* tx_w;
  const int* tx_deg;   // [5][nx]: entries in use
  const int* ty_col;   // [5][ny][kw]
  const float* ty_w;
  const int* ty_deg;   // [5][ny]
  float2* tmp;         // [25][nv] scratch between the x and y passes of the uniform S^T
  int periodic_x, periodic_y;
  int halo;            // largest |source - target| of the uniform transposed stencils (wrapped)
  // one-pass S^T: the transposed stencils dense by offset, [5][n][dw] weights of the sources
  // target + d, d in [-dhalo, dhalo] (the short way round), at d + dhalo
  const float* tx_dense;
  const float* ty_dense;
  int dhalo, dw;
  const long long* tm_ptr;  // [25][nv+1]
  const int* tm_col;
  const float* tm_w;
};
cudaError_t launch_adjoint_step(const AdjointArgs& a, cudaStream_t s);
// Ghost width of the pairs of the one-pass S^T (its largest transposed-stencil halo), and whether
// that kernel takes a uniform grid (halo, periodic axes at least two ghost widths long).
constexpr int kAdjGhost = 8;
bool adjoint_tma_usable(int nx, int ny, int periodic_x, int periodic_y, int halo);
// The halo the one-pass S^T is compiled for (4 or 8) given the stencils' halo, and the row width
// of its dense tables.
inline int adjoint_tma_halo(int halo) { return halo <= 4 ? 4 : 8; }
inline int adjoint_dense_width(int h) { return (2 * h + 1 + 3) / 4 * 4; }
struct InitVjpArgs {
  const double *rho, *u, *v, *T;
  const float* lam;
  float *du, *dv;
  long long nv;
  Consts cs;
  CollideK cp;
};
cudaError_t launch_init_vjp(const InitVjpArgs& a, cudaStream_t s);

}  // namespace sllbm
