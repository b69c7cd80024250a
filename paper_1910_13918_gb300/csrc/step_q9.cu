// SLLBM step on the D2Q9 velocity set, the standard set the paper compares D2Q25 with in the
// isothermal Taylor-Green study (Sec. III.A): the same pull streaming (Eq. sl_streaming), and
// BGK (Eq. streaming_fg) towards the same fourth-order equilibrium (Sec. II.A) evaluated at
// theta = 1 on the D1Q3 tensor-product nodes 0, +sqrt3, -sqrt3 (weights 2/3, 1/6, 1/6).  On those
// nodes He_3 vanishes and He_4 equals -3 He_2, so the expansion aliases onto lower orders: mass
// and momentum are exact, the third moment misses its u^3 term (the defect in Galilean
// invariance that the comparison shows).
//
// One population (the isothermal configuration) in planar storage, velocity i = 3a + b:
// FP32 / BF16 deviations f_i - w_i with FP32 arithmetic, or FP64 full populations.  Uniform
// grids in FP32 / BF16 run the tiled kernel below (shared-memory windows, sum factorisation);
// transformed grids, FP64, and uniform grids whose departures reach farther than its window run
// the gather kernel: one thread per vertex reads the (p+1)^2 stencil of each of the 9 planes
// through L1/L2 (per-axis tables, or the per-(velocity, vertex) cells and local coordinates).
#include <type_traits>

#include "kernels.h"
#include "tma.cuh"

namespace sllbm {

namespace {

constexpr int kN1 = 3;          // D1Q3
constexpr int kN = kN1 * kN1;   // D2Q9

template <typename Store>
__device__ __forceinline__ double ld_val(const Store* p) {
  if constexpr (std::is_same<Store, double>::value)
    return __ldg(p);
  else
    return (double)ld_store(p);
}

// Stencil of velocity i at vertex (ix, iy): first node column and row, and the 1D weights.
template <int P, bool Mapped, typename T>
__device__ __forceinline__ void stencil(const StepArgs& a, int i, long long v, int ix, int iy, int* sx,
                                        int* sy, T (&wx)[P + 1], T (&wy)[P + 1]) {
  const int ia = i / kN1, ib = i % kN1;
  if (Mapped) {
    const long long d = (long long)i * a.nv + v;
    *sx = a.dcx[d] * P;
    *sy = a.dcy[d] * P;
    if constexpr (std::is_same<T, double>::value) {
      lagrange_basis<P, double>(a.nodes, a.dr64[d], wx);
      lagrange_basis<P, double>(a.nodes, a.ds64[d], wy);
    } else {
      lagrange_basis<P, float>(a.nodesf, a.dr[d], wx);
      lagrange_basis<P, float>(a.nodesf, a.ds[d], wy);
    }
  } else {
    *sx = ix + a.offx[ia * a.nx + ix];
    *sy = iy + a.offy[ib * a.ny + iy];
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      if constexpr (std::is_same<T, double>::value) {
        wx[k] = a.wx64[(ia * a.nx + ix) * (P + 1) + k];
        wy[k] = a.wy64[(ib * a.ny + iy) * (P + 1) + k];
      } else {
        wx[k] = a.wx[(ia * a.nx + ix) * (P + 1) + k];
        wy[k] = a.wy[(ib * a.ny + iy) * (P + 1) + k];
      }
    }
  }
}

// Equilibrium at theta = 1 (q = 0, so A_k(u) = u^k): f_ab^eq = w_a w_b rho (1 + em1(a, b)) with
// em1(a, b) = sum_{(k,l) != (0,0), k+l <= 4} u_x^k he[k][a] u_y^l he[l][b].
template <typename T>
struct Eq9 {
  T X[4][kN1];   // u_x^k he[k][a], k = 1..4
  T S[5][kN1];   // sum_{l=1..m} u_y^l he[l][b]
};

template <typename T>
__device__ __forceinline__ void eq9_factors(const T (&he)[kQ1][kQ1], T ux, T uy, Eq9<T>& e) {
  const T ax[5] = {T(1), ux, ux * ux, ux * ux * ux, ux * ux * ux * ux};
  const T ay[5] = {T(1), uy, uy * uy, uy * uy * uy, uy * uy * uy * uy};
#pragma unroll
  for (int a = 0; a < kN1; ++a)
#pragma unroll
    for (int k = 1; k <= 4; ++k) e.X[k - 1][a] = ax[k] * he[k][a];
#pragma unroll
  for (int b = 0; b < kN1; ++b) {
    e.S[0][b] = T(0);
#pragma unroll
    for (int m = 1; m <= 4; ++m) e.S[m][b] = e.S[m - 1][b] + ay[m] * he[m][b];
  }
}

template <typename T>
__device__ __forceinline__ T eq9_em1(const Eq9<T>& e, int a, int b) {
  T s = e.S[4][b];
#pragma unroll
  for (int k = 1; k <= 4; ++k) s += e.X[k - 1][a] * (T(1) + e.S[4 - k][b]);
  return s;
}

// BGK of one vertex in deviation form, FP32: fb[i] = f_i - w_i before, the post-collision
// deviations after.  Returns false if the density is non-positive or a value is not finite.
__device__ __forceinline__ bool collide_q9_f32(float (&fb)[kN], const Consts& cs, const CollideK& cp) {
  float drho = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
  for (int i = 0; i < kN; ++i) {   // sum w = 1 and sum w xi = 0: the moments of fbar
    drho += fb[i];
    jx += fb[i] * cs.xif[i / kN1];
    jy += fb[i] * cs.xif[i % kN1];
  }
  const float rho = 1.f + drho;
  const float ux = jx / rho, uy = jy / rho;
  Eq9<float> e;
  eq9_factors<float>(cs.hef, ux, uy, e);
  const float om = cp.omegaf;
  // relax, and sum the residual moments of (f^eq - f) to restore mass and momentum to the
  // rounding of those sums (as in the D2Q25 kernels)
  float r0 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
  for (int i = 0; i < kN; ++i) {
    const int ia = i / kN1, ib = i % kN1;
    const float w = cs.wf[ia] * cs.wf[ib];
    const float d = w * (drho + rho * eq9_em1<float>(e, ia, ib)) - fb[i];
    r0 += d;
    r1 += d * cs.xif[ia];
    r2 += d * cs.xif[ib];
    fb[i] = fmaf(om, d, fb[i]);
  }
  // remove om (r0 + r1 xi_x + r2 xi_y) w_i: sum w = 1, sum w xi xi = I on D2Q9
#pragma unroll
  for (int i = 0; i < kN; ++i) {
    const int ia = i / kN1, ib = i % kN1;
    const float w = cs.wf[ia] * cs.wf[ib];
    fb[i] -= om * w * (r0 + r1 * cs.xif[ia] + r2 * cs.xif[ib]);
  }
  return rho > 0.f && isfinite(rho) && isfinite(ux) && isfinite(uy);
}

template <int P, typename Store, bool Mapped>
__global__ void __launch_bounds__(128) step_q9_kernel(const __grid_constant__ StepArgs a) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= a.nv) return;
  const int ix = (int)(v % a.nx), iy = (int)(v / a.nx);
  const Store* src = static_cast<const Store*>(a.src);
  Store* dst = static_cast<Store*>(a.dst);
  const size_t o = (size_t)iy * a.pitch + ix;
  constexpr bool F64 = std::is_same<Store, double>::value;

  if constexpr (F64) {
    // full populations: sum_{a,b} psi_a psi_b f(node(a, b)), moments, BGK
    double f[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      int sx, sy;
      double wx[P + 1], wy[P + 1];
      stencil<P, Mapped, double>(a, i, v, ix, iy, &sx, &sy, wx, wy);
      const Store* pl = src + (size_t)i * a.plane_stride;
      double acc = 0.0;
#pragma unroll
      for (int kb = 0; kb <= P; ++kb) {
        const size_t r = (size_t)wrap_index(sy + kb, a.ny, a.periodic_y) * a.pitch;
        double ax = 0.0;
#pragma unroll
        for (int ka = 0; ka <= P; ++ka) ax += wx[ka] * ld_val(pl + r + wrap_index(sx + ka, a.nx, a.periodic_x));
        acc += wy[kb] * ax;
      }
      f[i] = acc;
    }
    double rho = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      rho += f[i];
      jx += f[i] * a.cs.xi[i / kN1];
      jy += f[i] * a.cs.xi[i % kN1];
    }
    const double ux = jx / rho, uy = jy / rho;
    Eq9<double> e;
    eq9_factors<double>(a.cs.he, ux, uy, e);
    const double om = a.cp.omega;
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      const int ia = i / kN1, ib = i % kN1;
      const double feq = a.cs.w[ia] * a.cs.w[ib] * rho * (1.0 + eq9_em1<double>(e, ia, ib));
      dst[(size_t)i * a.plane_stride + o] = f[i] - om * (f[i] - feq);
    }
    if (!(rho > 0.0 && isfinite(rho))) atomicOr(a.flag, 1);
  } else {
    // deviations fbar = f - w, FP32; interpolation in difference form (constants exact)
    float fb[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      int sx, sy;
      float wx[P + 1], wy[P + 1];
      stencil<P, Mapped, float>(a, i, v, ix, iy, &sx, &sy, wx, wy);
      const Store* pl = src + (size_t)i * a.plane_stride;
      int col[P + 1];
#pragma unroll
      for (int k = 0; k <= P; ++k) col[k] = wrap_index(sx + k, a.nx, a.periodic_x);
      float rows[P + 1];
#pragma unroll
      for (int kb = 0; kb <= P; ++kb) {
        const Store* r = pl + (size_t)wrap_index(sy + kb, a.ny, a.periodic_y) * a.pitch;
        const float base = ld_store(r + col[0]);
        float acc = base;
#pragma unroll
        for (int ka = 1; ka <= P; ++ka) acc = fmaf(wx[ka], ld_store(r + col[ka]) - base, acc);
        rows[kb] = acc;
      }
      float acc = rows[0];
#pragma unroll
      for (int kb = 1; kb <= P; ++kb) acc = fmaf(wy[kb], rows[kb] - rows[0], acc);
      fb[i] = acc;
    }
    const bool ok = collide_q9_f32(fb, a.cs, a.cp);
#pragma unroll
    for (int i = 0; i < kN; ++i) st_store(dst + (size_t)i * a.plane_stride + o, fb[i]);
    if (!ok) atomicOr(a.flag, 1);
  }
}

// Uniform grids, FP32 arithmetic: tiles of 32 x kTY vertices, one thread each.  Plane by plane,
// the source window that the tile's stencils reach is staged in shared memory (coalesced loads;
// the next plane's window is loaded into registers while the current one is interpolated), then
// interpolated along y for every staged column with the taps of the tile row (warp r takes row
// r), and along x for every vertex with its own taps: the sum factorisation of the
// tensor-product stencil, 2(p+1) taps a value instead of (p+1)^2.  The source offsets of the
// staged elements do not depend on the plane and are formed once per tile.
constexpr int kTY = 8;                 // tile rows
constexpr int kNT = 32 * kTY;          // threads: warp r handles tile row r
constexpr int kRC = 3;                 // window row chunks: row r of the window is read by warp r % kTY
constexpr int kCC = 3;                 // window column chunks of 32
constexpr int kMaxW = 32 * kCC, kMaxH = kTY * kRC;

struct Window {
  int ox, oy;   // window origin relative to the tile origin (the smallest stencil offsets)
  int W, H;     // window columns (<= kMaxW) and rows (<= kMaxH)
};

template <int P, typename Store>
__global__ void __launch_bounds__(kNT) step_q9_tiled_kernel(const __grid_constant__ StepArgs a,
                                                             const Window win) {
  __shared__ float S[kMaxH * kMaxW];   // staged window of one plane, [H][W]
  __shared__ float T[kTY * kMaxW];     // y-interpolated rows, [kTY][W]
  const int tid = threadIdx.x, lane = tid & 31, row = tid >> 5;
  const int tiles_x = (a.nx + 31) / 32;
  const int tx0 = (int)(blockIdx.x % tiles_x) * 32, ty0 = (int)(blockIdx.x / tiles_x) * kTY;
  const int x = tx0 + lane, y = ty0 + row;
  const int W = win.W, H = win.H;
  const Store* src = static_cast<const Store*>(a.src);

  // taps of this thread's column (x pass) and of its warp's row (y pass), clamped into the grid
  // for threads past its edge; stencil starts as window column / row
  const int xc = min(x, a.nx - 1), yc = min(y, a.ny - 1);
  int xo[kN1], yo[kN1];
  float xw[kN1][P + 1], yw[kN1][P + 1];
#pragma unroll
  for (int c = 0; c < kN1; ++c) {
    xo[c] = xc + a.offx[c * a.nx + xc] - tx0 - win.ox;
    yo[c] = yc + a.offy[c * a.ny + yc] - ty0 - win.oy;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      xw[c][k] = a.wx[(size_t)(c * a.nx + xc) * (P + 1) + k];
      yw[c][k] = a.wy[(size_t)(c * a.ny + yc) * (P + 1) + k];
    }
  }
  // the window elements this thread stages: rows row + kTY j, columns lane + 32 m (wrapped or
  // clamped into the grid), as offsets within a plane
  size_t grow[kRC];
  int gcol[kCC];
#pragma unroll
  for (int j = 0; j < kRC; ++j) {
    int gy = ty0 + win.oy + row + kTY * j;
    gy = a.periodic_y ? wrap_index(gy, a.ny, 1) : min(max(gy, 0), a.ny - 1);
    grow[j] = (size_t)gy * a.pitch;
  }
#pragma unroll
  for (int m = 0; m < kCC; ++m) {
    int gx = tx0 + win.ox + lane + 32 * m;
    gx = a.periodic_x ? wrap_index(gx, a.nx, 1) : min(max(gx, 0), a.nx - 1);
    gcol[m] = gx;
  }
  float pre[kRC][kCC];
  auto load = [&](int i) {
    const Store* pl = src + (size_t)i * a.plane_stride;
#pragma unroll
    for (int j = 0; j < kRC; ++j)
#pragma unroll
      for (int m = 0; m < kCC; ++m)
        if (row + kTY * j < H && lane + 32 * m < W) pre[j][m] = ld_store(pl + grow[j] + gcol[m]);
  };
  load(0);
  float fb[kN];
#pragma unroll
  for (int i = 0; i < kN; ++i) {
    const int ca = i / kN1, cb = i % kN1;
    // S is free: every thread is past the previous plane's y pass (second barrier below)
#pragma unroll
    for (int j = 0; j < kRC; ++j)
#pragma unroll
      for (int m = 0; m < kCC; ++m)
        if (row + kTY * j < H && lane + 32 * m < W) S[(row + kTY * j) * W + lane + 32 * m] = pre[j][m];
    if (i + 1 < kN) load(i + 1);
    __syncthreads();   // window staged; every thread is past the previous plane's x pass (T free)
#pragma unroll
    for (int m = 0; m < kCC; ++m) {
      const int c = lane + 32 * m;
      if (c < W) {
        const float* col = S + yo[cb] * W + c;
        const float base = col[0];
        float acc = base;
#pragma unroll
        for (int k = 1; k <= P; ++k) acc = fmaf(yw[cb][k], col[k * W] - base, acc);
        T[row * W + c] = acc;
      }
    }
    __syncthreads();   // T complete
    {
      const float* t = T + row * W + xo[ca];
      const float base = t[0];
      float acc = base;
#pragma unroll
      for (int k = 1; k <= P; ++k) acc = fmaf(xw[ca][k], t[k] - base, acc);
      fb[i] = acc;
    }
  }
  if (x >= a.nx || y >= a.ny) return;
  const bool ok = collide_q9_f32(fb, a.cs, a.cp);
  Store* dst = static_cast<Store*>(a.dst) + (size_t)y * a.pitch + x;
#pragma unroll
  for (int i = 0; i < kN; ++i) st_store(dst + (size_t)i * a.plane_stride, fb[i]);
  if (!ok) atomicOr(a.flag, 1);
}

// FP32 storage: the same tile, with the windows of all 9 planes requested up front by
// asynchronous 4-byte copies into shared memory (one commit group per plane), so that the
// interpolation of plane i overlaps the transfer of the later planes.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until the copies of plane i (group i of 9) have landed
__device__ __forceinline__ void cp_async_wait_plane(int i) {
  switch (i) {
    case 0: asm volatile("cp.async.wait_group 8;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    case 7: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
  }
}

size_t async_smem_bytes(const Window& w) { return sizeof(float) * ((size_t)kN * w.H * w.W + (size_t)kTY * w.W); }

template <int P>
__global__ void __launch_bounds__(kNT) step_q9_async_kernel(const __grid_constant__ StepArgs a,
                                                             const Window win) {
  extern __shared__ float q9_smem[];
  const int W = win.W, H = win.H;
  float* S = q9_smem;              // [9][H][W] staged windows
  float* T = S + kN * H * W;       // [kTY][W] y-interpolated rows
  const int tid = threadIdx.x, lane = tid & 31, row = tid >> 5;
  const int tiles_x = (a.nx + 31) / 32;
  const int tx0 = (int)(blockIdx.x % tiles_x) * 32, ty0 = (int)(blockIdx.x / tiles_x) * kTY;
  const int x = tx0 + lane, y = ty0 + row;
  const float* src = static_cast<const float*>(a.src);
  {
    size_t grow[kRC];
    int gcol[kCC];
#pragma unroll
    for (int j = 0; j < kRC; ++j) {
      int gy = ty0 + win.oy + row + kTY * j;
      gy = a.periodic_y ? wrap_index(gy, a.ny, 1) : min(max(gy, 0), a.ny - 1);
      grow[j] = (size_t)gy * a.pitch;
    }
#pragma unroll
    for (int m = 0; m < kCC; ++m) {
      int gx = tx0 + win.ox + lane + 32 * m;
      gx = a.periodic_x ? wrap_index(gx, a.nx, 1) : min(max(gx, 0), a.nx - 1);
      gcol[m] = gx;
    }
#pragma unroll 1
    for (int i = 0; i < kN; ++i) {
      const float* pl = src + (size_t)i * a.plane_stride;
      float* Si = S + i * H * W;
#pragma unroll
      for (int j = 0; j < kRC; ++j)
#pragma unroll
        for (int m = 0; m < kCC; ++m)
          if (row + kTY * j < H && lane + 32 * m < W)
            cp_async4(Si + (row + kTY * j) * W + lane + 32 * m, pl + grow[j] + gcol[m]);
      cp_async_commit();
    }
  }
  const int xc = min(x, a.nx - 1), yc = min(y, a.ny - 1);
  int xo[kN1], yo[kN1];
  float xw[kN1][P + 1], yw[kN1][P + 1];
#pragma unroll
  for (int c = 0; c < kN1; ++c) {
    xo[c] = xc + a.offx[c * a.nx + xc] - tx0 - win.ox;
    yo[c] = yc + a.offy[c * a.ny + yc] - ty0 - win.oy;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      xw[c][k] = a.wx[(size_t)(c * a.nx + xc) * (P + 1) + k];
      yw[c][k] = a.wy[(size_t)(c * a.ny + yc) * (P + 1) + k];
    }
  }
  float fb[kN];
#pragma unroll
  for (int i = 0; i < kN; ++i) {
    const int ca = i / kN1, cb = i % kN1;
    cp_async_wait_plane(i);
    __syncthreads();   // plane i staged by every thread; every thread is past the previous x pass
    const float* Si = S + i * H * W;
#pragma unroll
    for (int m = 0; m < kCC; ++m) {
      const int c = lane + 32 * m;
      if (c < W) {
        const float* col = Si + yo[cb] * W + c;
        const float base = col[0];
        float acc = base;
#pragma unroll
        for (int k = 1; k <= P; ++k) acc = fmaf(yw[cb][k], col[k * W] - base, acc);
        T[row * W + c] = acc;
      }
    }
    __syncthreads();   // T complete
    {
      const float* t = T + row * W + xo[ca];
      const float base = t[0];
      float acc = base;
#pragma unroll
      for (int k = 1; k <= P; ++k) acc = fmaf(xw[ca][k], t[k] - base, acc);
      fb[i] = acc;
    }
  }
  if (x >= a.nx || y >= a.ny) return;
  const bool ok = collide_q9_f32(fb, a.cs, a.cp);
  float* dst = static_cast<float*>(a.dst) + (size_t)y * a.pitch + x;
#pragma unroll
  for (int i = 0; i < kN; ++i) dst[(size_t)i * a.plane_stride] = fb[i];
  if (!ok) atomicOr(a.flag, 1);
}

// FP32 or BF16 storage on uniform grids, persistent CTAs with Tensor Memory Accelerator staging:
// a tile's window of the 9 planes arrives as three tensor copies (cp.async.bulk.tensor, 3 planes
// each, one mbarrier each), issued a whole tile ahead into the other of two buffers, so that the
// copies of the next tile overlap the interpolation and collision of this one, and plane i's
// interpolation waits only for its own group.  The state's ghost cells hold the periodic images
// (every write stores them too), so a window never wraps; its origin is rounded down to a
// 16-byte boundary and the stencil offsets carry the remainder.  The interpolation runs in FP32
// on the staged values of either storage type.
constexpr int kQ9Groups = 3;   // tensor copies per tile (3 planes each)

struct Q9Tma {
  CUtensorMap tmap;   // 3D: (column, row, plane) over the whole allocation, in the storage type
  int oxa;            // window origin relative to the tile origin, rounded down to 16 bytes
  int Wa, H;          // window columns (a multiple of 16 bytes) and rows
  int dx;             // ox - oxa: shift of the stencil offsets
};

// elements (of elem bytes) of one copy group (3 planes of H x Wa), padded to keep every copy
// 128-byte aligned
__host__ __device__ inline int q9_group_elems(int Wa, int H, int elem) {
  return (3 * H * Wa * elem + 127) / 128 * 128 / elem;
}

size_t q9_tma_smem_bytes(int Wa, int H, int elem) {
  return 128 + (size_t)elem * 2 * kQ9Groups * q9_group_elems(Wa, H, elem) + sizeof(float) * (size_t)kTY * Wa +
         sizeof(uint64_t) * 2 * kQ9Groups;
}

__device__ __forceinline__ float q9_lds(const float* p) { return *p; }
__device__ __forceinline__ float q9_lds(const __nv_bfloat16* p) { return __bfloat162float(*p); }

template <int P, typename Store>
__global__ void __launch_bounds__(kNT) step_q9_tma_kernel(const __grid_constant__ StepArgs a,
                                                           const __grid_constant__ Window win,
                                                           const __grid_constant__ Q9Tma qt) {
  extern __shared__ unsigned char q9t_smem[];
  Store* base = reinterpret_cast<Store*>(q9t_smem + ((128 - (smem_u32(q9t_smem) & 127)) & 127));
  const int W4 = qt.Wa, H = qt.H;
  const int plane_elems = H * W4, group_elems = q9_group_elems(W4, H, (int)sizeof(Store)),
            buf_elems = kQ9Groups * group_elems;
  Store* S = base;                                              // [2][3 groups][3][H][W4]
  float* T = reinterpret_cast<float*>(S + 2 * buf_elems);       // [kTY][W4]
  uint64_t* BAR = reinterpret_cast<uint64_t*>(T + kTY * W4);   // [2][3]; offset a multiple of 8 B
  const int tid = threadIdx.x, lane = tid & 31, row = tid >> 5;
  const int tiles_x = (a.nx + 31) / 32;
  const int ntiles = tiles_x * ((a.ny + kTY - 1) / kTY);
  if (tid == 0) {
    for (int k = 0; k < 2 * kQ9Groups; ++k) mbar_init(&BAR[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int tile, int buf) {
    if (tid != 0 || tile >= ntiles) return;
    const int tx0 = (tile % tiles_x) * 32, ty0 = (tile / tiles_x) * kTY;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
#pragma unroll
    for (int g = 0; g < kQ9Groups; ++g) {
      uint64_t* bar = &BAR[buf * kQ9Groups + g];
      mbar_expect_tx(bar, (unsigned)(sizeof(Store) * 3 * plane_elems));
      tma_load_3d(S + (size_t)buf * buf_elems + (size_t)g * group_elems, &qt.tmap, a.gx + tx0 + qt.oxa,
                  a.gy + ty0 + win.oy, 3 * g, bar);
    }
  };
  issue(blockIdx.x, 0);
  const int my_tiles = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
#pragma unroll 1
  for (int k = 0; k < my_tiles; ++k) {
    const int tile = blockIdx.x + k * gridDim.x, buf = k & 1;
    const unsigned parity = (unsigned)((k >> 1) & 1);
    const int tx0 = (tile % tiles_x) * 32, ty0 = (tile / tiles_x) * kTY;
    const int x = tx0 + lane, y = ty0 + row;
    __syncthreads();   // every thread is past tile k - 1: its buffer (the other one) is free
    issue(tile + gridDim.x, buf ^ 1);
    // taps of this thread's column (x pass) and of its warp's row (y pass), clamped into the grid
    // for threads past its edge; stencil starts as window column / row
    const int xc = min(x, a.nx - 1), yc = min(y, a.ny - 1);
    int xo[kN1], yo[kN1];
    float xw[kN1][P + 1], yw[kN1][P + 1];
#pragma unroll
    for (int c = 0; c < kN1; ++c) {
      xo[c] = xc + a.offx[c * a.nx + xc] - tx0 - win.ox + qt.dx;
      yo[c] = yc + a.offy[c * a.ny + yc] - ty0 - win.oy;
#pragma unroll
      for (int q = 0; q <= P; ++q) {
        xw[c][q] = a.wx[(size_t)(c * a.nx + xc) * (P + 1) + q];
        yw[c][q] = a.wy[(size_t)(c * a.ny + yc) * (P + 1) + q];
      }
    }
    const Store* Sb = S + (size_t)buf * buf_elems;
    float fb[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) {
      const int ca = i / kN1, cb = i % kN1;
      // group landed (every thread then also past the previous plane's x pass: T free); if the
      // wait ran out, every thread stops together after the copies still in flight
      const bool late = (i % 3 == 0) && !mbar_wait(&BAR[buf * kQ9Groups + i / 3], parity, a.flag);
      if (__syncthreads_or(late)) {
        for (int g = i / 3; g < kQ9Groups; ++g)   // this group (it may still land) and the later ones
          if (!mbar_wait(&BAR[buf * kQ9Groups + g], parity, a.flag)) return;
        if (k + 1 < my_tiles)                          // the next tile's groups
          for (int g = 0; g < kQ9Groups; ++g)
            if (!mbar_wait(&BAR[(buf ^ 1) * kQ9Groups + g], (unsigned)(((k + 1) >> 1) & 1), a.flag)) return;
        return;
      }
      const Store* Si = Sb + (i / 3) * group_elems + (i % 3) * plane_elems;
#pragma unroll
      for (int m = 0; m < kCC; ++m) {
        const int c = lane + 32 * m;
        if (c < W4) {
          const Store* col = Si + yo[cb] * W4 + c;
          const float b0 = q9_lds(col);
          float acc = b0;
#pragma unroll
          for (int q = 1; q <= P; ++q) acc = fmaf(yw[cb][q], q9_lds(col + q * W4) - b0, acc);
          T[row * W4 + c] = acc;
        }
      }
      __syncthreads();   // T complete
      {
        const float* t = T + row * W4 + xo[ca];
        const float b0 = t[0];
        float acc = b0;
#pragma unroll
        for (int q = 1; q <= P; ++q) acc = fmaf(xw[ca][q], t[q] - b0, acc);
        fb[i] = acc;
      }
    }
    if (x < a.nx && y < a.ny) {
      const bool ok = collide_q9_f32(fb, a.cs, a.cp);
      if (!ok) atomicOr(a.flag, 1);
      Store* dst = static_cast<Store*>(a.dst);
      store_images(a.ghost, x, y, [&](int xx, int yy) {
        Store* o = dst + (ptrdiff_t)yy * a.pitch + xx;
#pragma unroll
        for (int i = 0; i < kN; ++i) st_store(o + (size_t)i * a.plane_stride, fb[i]);
      });
    }
  }
}

// Window of the TMA kernel for a uniform grid and elements of elem bytes, or false if the kernel
// cannot take it (the window, rounded to 16-byte columns, must fit the shared memory and stay
// inside the ghost cells).
bool q9_tma_window(const StepArgs& a, int elem, Window* win, Q9Tma* qt) {
  if (a.mapped || a.xs != 1 || (elem != 4 && elem != 2)) return false;
  const int u = 16 / elem;   // columns of 16 bytes
  *win = Window{a.offx_min, a.offy_min, 32 + a.offx_max - a.offx_min, kTY + a.offy_max - a.offy_min};
  const int oxa = (win->ox >= 0) ? win->ox / u * u : -((-win->ox + u - 1) / u * u);
  qt->oxa = oxa;
  qt->dx = win->ox - oxa;
  qt->Wa = (win->W + qt->dx + u - 1) / u * u;
  qt->H = win->H;
  if (qt->Wa > kMaxW || qt->H > kMaxH || qt->H > 256) return false;
  // first and last window column / row of any tile, against the allocation's ghost cells
  const int tiles_x = (a.nx + 31) / 32, tiles_y = (a.ny + kTY - 1) / kTY;
  if (oxa < -a.gx || (tiles_x - 1) * 32 + oxa + qt->Wa > a.pitch - a.gx) return false;
  if (win->oy < -a.gy || (tiles_y - 1) * kTY + win->oy + qt->H > a.rows_alloc - a.gy) return false;
  if ((a.gx * elem) % 16 != 0 || ((size_t)a.pitch * elem) % 16 != 0) return false;   // 16-byte copy origins
  return q9_tma_smem_bytes(qt->Wa, qt->H, elem) <= 200 * 1024;
}

template <int P, typename Store>
static cudaError_t launch_q9_tma(const StepArgs& a, const Window& win, Q9Tma qt, cudaStream_t s) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const Store* alloc = static_cast<const Store*>(a.src) - ((ptrdiff_t)a.gy * a.pitch + a.gx);
  const cuuint64_t dims[3] = {(cuuint64_t)a.pitch, (cuuint64_t)a.rows_alloc, (cuuint64_t)kN};
  const cuuint64_t strides[2] = {(cuuint64_t)a.pitch * sizeof(Store), (cuuint64_t)a.plane_stride * sizeof(Store)};
  const cuuint32_t box[3] = {(cuuint32_t)qt.Wa, (cuuint32_t)qt.H, 3u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUtensorMapDataType dt =
      sizeof(Store) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (enc(&qt.tmap, dt, 3, const_cast<Store*>(alloc), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  auto kern = step_q9_tma_kernel<P, Store>;
  const size_t smem = q9_tma_smem_bytes(qt.Wa, qt.H, (int)sizeof(Store));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, n_sm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kNT, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ntiles = ((a.nx + 31) / 32) * ((a.ny + kTY - 1) / kTY);
  const int grid = ntiles < n_sm * per_sm ? ntiles : n_sm * per_sm;   // persistent CTAs
  kern<<<grid, kNT, smem, s>>>(a, win, qt);
  return cudaGetLastError();
}

template <int P, typename Store>
cudaError_t launch_ps(const StepArgs& a, cudaStream_t s) {
  if constexpr (!std::is_same<Store, double>::value) {
    if (a.q9_tma) {   // chosen (and the ghost images kept) by the host set-up
      Window win;
      Q9Tma qt;
      if (!q9_tma_window(a, (int)sizeof(Store), &win, &qt)) return cudaErrorNotSupported;
      return launch_q9_tma<P, Store>(a, win, qt, s);
    }
  }
  if constexpr (!std::is_same<Store, double>::value) {
    // uniform grid whose stencil window fits the staging buffer: the tiled kernel
    const Window win{a.offx_min, a.offy_min, 32 + a.offx_max - a.offx_min, kTY + a.offy_max - a.offy_min};
    if (!a.mapped && win.W <= kMaxW && win.H <= kMaxH) {
      const unsigned tiles = (unsigned)(((a.nx + 31) / 32) * ((a.ny + kTY - 1) / kTY));
      if constexpr (std::is_same<Store, float>::value) {
        const size_t smem = async_smem_bytes(win);
        if (smem > 48 * 1024) {   // wide windows need more than the default dynamic shared memory
          const cudaError_t e = cudaFuncSetAttribute(step_q9_async_kernel<P>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
          if (e != cudaSuccess) return e;
        }
        step_q9_async_kernel<P><<<tiles, kNT, smem, s>>>(a, win);
      } else {
        step_q9_tiled_kernel<P, Store><<<tiles, kNT, 0, s>>>(a, win);
      }
      return cudaGetLastError();
    }
  }
  const int threads = 128;
  const unsigned blocks = (unsigned)((a.nv + threads - 1) / threads);
  if (a.mapped)
    step_q9_kernel<P, Store, true><<<blocks, threads, 0, s>>>(a);
  else
    step_q9_kernel<P, Store, false><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename Store>
cudaError_t launch_store(const StepArgs& a, cudaStream_t s) {
  switch (a.P) {
    case 1: return launch_ps<1, Store>(a, s);
    case 2: return launch_ps<2, Store>(a, s);
    case 3: return launch_ps<3, Store>(a, s);
    case 4: return launch_ps<4, Store>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool q9_tma_usable(const StepArgs& a, int elem) {
  Window win;
  Q9Tma qt;
  return q9_tma_window(a, elem, &win, &qt);
}

cudaError_t launch_step_q9(const StepArgs& a, int store, cudaStream_t s) {
  if (a.cs.nq1 != kN1 || a.cp.npop != 1 || a.xs != 1 || a.nv == 0) return cudaErrorInvalidValue;
  switch (store) {
    case kStoreF32: return launch_store<float>(a, s);
    case kStoreBF16: return launch_store<__nv_bfloat16>(a, s);
    case kStoreF64: return launch_store<double>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sllbm
