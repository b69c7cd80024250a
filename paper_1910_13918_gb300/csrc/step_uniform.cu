// Fused SLLBM step for uniform grids, FP32 arithmetic, FP32 or BF16 deviation storage.
//
// Pull streaming (Eq. sl_streaming) + moments + fourth-order equilibrium + BGK (Eq. streaming_fg,
// Pr = 1) in one kernel.  On a uniform grid the departure x_v - dt xi_i separates per axis and,
// away from clamped (zero-gradient) boundaries, repeats with the period p of the cells: the
// stencil offset and Lagrange weights of vertex j depend only on the velocity component and on
// the local node j mod p.  The kernel uses that "pattern" (per component and local node: a start
// offset in [-p, 0] and p+1 weights), for the y interpolation of every staged column and the x
// interpolation of every vertex.  Vertices whose table entries differ from the pattern (next to
// zero-gradient boundaries) are not written here; the host runs the gather kernel on exactly
// those vertices afterwards.
//
// State: f and g share the departure points, so the state interleaves them ((f, g) pairs per
// velocity plane and vertex) and every interpolation step moves and combines the pair at once:
// 64-bit shared-memory and global accesses, packed FP32x2 FMAs.
//
// Persistent CTAs (two per SM) walk over tiles of 32 x TY
// vertices (TY a multiple of p), one vertex per thread.  The 25 pair planes of a tile are done in
// 5 stages, one per x component a.  A stage (the 5 planes b = 0..4) is copied into shared memory by one TMA tensor copy (tile +
// stencil halo; the state layout carries ghost cells with the periodic images, so a tile never
// wraps), completing on an mbarrier, three stages ahead in four buffers.  Phase k runs the y pass
// of stage k (task = plane b, staged column, chunk of rows: register window of the column) and
// the x pass of stage k-1 (thread = vertex): five barriers per tile.  After stage 4 every thread
// holds the 50 pre-collision deviations of its vertex, collides in registers and writes 25
// coalesced rows of pairs (plus periodic images in the ghost cells), in the phase that runs the
// y pass of the next tile's first stage.
//
// Interpolation form: sum_alpha w_alpha v_{s+alpha} is evaluated as
//   v_s + sum_{alpha >= 1} W_alpha (v_{s+alpha} - v_{s+alpha-1}),  W_alpha = sum_{beta >= alpha} w_beta,
// equal to it because the weights sum to one.  A constant field is reproduced exactly in FP32
// (with the FP32-rounded weights themselves the deficit of their sum would bias every uniform
// region the same way every step, a systematic mass drift), and in the y pass the differences of
// a staged column are formed once and shared by all the rows that read them.
#include <atomic>

#include "kernels.h"
#include "tma.cuh"

namespace sllbm {

namespace {

// Stencils of the pattern.  The stencil of a departure point is the cell that contains it, so it
// starts on a cell boundary; with the offset D in [-p, 0] of the start relative to the vertex this
// leaves, for the vertex at local node l of its cell, D = -l (own cell) or, at l = 0 only,
// D = -p (the cell before).  (The host checks the tables for exactly this form.)  Staged rows
// therefore reach from y0 - p (D = -p at the tile's first row) to y0 + TY (the last cell of the
// tile), and the start row of every stencil is a cell boundary.
//
// Tile of 32 x TY vertices, TY = 8 (6 for p = 3), two CTAs of 32 TY threads per SM: one CTA's
// barriers and collision burst overlap the other's interpolation (one CTA of twice the rows per
// SM measured slower at p = 3 and 4).  A y-pass task covers RC = TY / NH rows of one staged
// column (NH = 1: the whole column), from a window of RW = RC + p + 1 rows.
template <int P>
struct TileShape {
  static constexpr int TY = (P == 3) ? 6 : 8;
  static constexpr int NT = 32 * TY;
  static constexpr int MINB = 2;                 // CTAs per SM
  static constexpr int R = TY + P + 1;           // staged rows y0-P .. y0+TY
  static constexpr int NH = 1;                   // row chunks per staged column
  static constexpr int RC = TY / NH;             // rows per y-pass task (a multiple of P)
  static constexpr int RW = RC + P + 1;          // window rows per y-pass task
  static_assert(RC % P == 0, "row chunks must hold whole periods of the pattern");
};

constexpr int kStageBuffers = 4;   // TMA staging buffers per CTA (prefetch distance 3 stages)
constexpr int kCO = 4;             // staged column origin x0 - 4: 16-byte aligned for both pair types
constexpr int kC = 32 + 2 * kCO;   // staged columns
// Rows of the y-pass output T keep column c at a skewed position: the lanes of one cell read the
// same columns and cells are P columns apart, so plain rows would put several cells on one
// shared-memory bank.  With a gap every 16 columns (P = 4, 2, 1) or two every 17 (P = 3) the
// x-pass reads of each tap and the y-pass row stores are free of bank conflicts.
template <int P>
__host__ __device__ constexpr int tpos(int c) {
  return P == 3 ? c + 2 * (c / 17) : (P == 1 ? c + (c >> 4) : c + 2 * (c >> 4));
}
template <int P>
struct TRow { static constexpr int N = tpos<P>(kC - 1) + 1; };   // T row length (pairs)
// ints of the DX [5][P] and EY [5] tables, rounded up to keep the mbarriers 8-byte aligned
__host__ __device__ constexpr int table_ints(int P) { return (kQ1 * P + kQ1 + 1) / 2 * 2; }

// Elements of one TMA box (5 planes x R rows x C columns x 2 populations), padded to 128 bytes.
template <int P, typename Store>
struct BoxShape {
  static constexpr int ELEMS = 5 * TileShape<P>::R * kC * 2;
  static constexpr int BYTES = ELEMS * (int)sizeof(Store);
  static constexpr int STRIDE = ((BYTES + 127) / 128) * 128 / (int)sizeof(Store);
};

// The P tail-sum taps of one (component, local node), stored as 4 (f, g) pairs (32 bytes,
// 16-byte aligned): two 16-byte loads.
template <int P>
__device__ __forceinline__ void load_taps(const float2* w, float2 (&W)[P]) {
  const float4 q0 = *reinterpret_cast<const float4*>(w);
  W[0] = make_float2(q0.x, q0.y);
  if (P > 1) W[1] = make_float2(q0.z, q0.w);
  if (P > 2) {
    const float4 q1 = *reinterpret_cast<const float4*>(w + 2);
    W[2 < P ? 2 : 0] = make_float2(q1.x, q1.y);
    if (P > 3) W[3 < P ? 3 : 0] = make_float2(q1.z, q1.w);
  }
}

// y interpolation of the RC rows of a task.  Window row j is task row j - P; row rr = m p + l
// has its stencil in cell m + e of the window (rows (m + e) p .. (m + e + 1) p), e = 1 except
// at l = 0 when the plane's departures fall in the cell before (E0 = false).  Straight-line code:
// the RC outputs are independent and interleave freely.
template <int P, int RC, int RW, bool E0>
__device__ __forceinline__ void y_rows(const float2 (&win)[RW], const float2 (&dl)[RW - 1],
                                       const float2 (&W)[P][P], float2* __restrict__ tout) {
#pragma unroll
  for (int rr = 0; rr < RC; ++rr) {
    const int l = rr % P, m = rr / P;
    const int s = (m + ((l == 0 && !E0) ? 0 : 1)) * P;
    float2 acc = win[s];
#pragma unroll
    for (int al = 1; al <= P; ++al) acc = fma2(W[l][al - 1], dl[s + al - 1], acc);
    tout[rr * TRow<P>::N] = acc;
  }
}

// y pass: task = (plane b, row chunk h, staged column c).  The first 5*NH*32 tasks give each
// warp one (b, h) and 32 columns; the right-hand 2P columns of the NH chunks of a plane b go to
// one more warp per b (NH*2P of its lanes) when the block has the warps, so that the branch on
// the plane's cell choice never diverges; otherwise they are packed.  A block never has more
// tasks than threads, so a thread's task is the same in every stage: it is set up once.
struct YTask {
  int src;    // element offset of the task's first window row in a staging buffer
  int dst;    // pair offset of its first output in a T buffer
  int b;      // plane (y component)
};

template <int P>
__device__ __forceinline__ bool y_task(int t, YTask& yt) {
  using TS = TileShape<P>;
  constexpr int TY = TS::TY, R = TS::R, NH = TS::NH, RC = TS::RC, NT = TS::NT;
  // The x pass reads staged columns [4 - P, 36 + P) only (stencil starts in [-P, 0] from the
  // column, P + 1 taps): 32 columns per plane in the warp tasks, the 2P others in the packed ones.
  constexpr int C0 = kCO - P;
  constexpr int CR = 2 * P;
  static_assert(NH * CR <= 32, "right-hand columns of one plane must fit in a warp");
  constexpr bool kSpread = kQ1 * (NH + 1) * 32 <= NT;
  constexpr int kTasks = kSpread ? kQ1 * (NH + 1) * 32 : kQ1 * NH * (32 + CR);
  static_assert(kTasks <= NT, "one y-pass task per thread at most");
  if (t >= kTasks) return false;
  int b, h, c;
  if (t < kQ1 * NH * 32) {
    const int g = t >> 5;
    b = g / NH;
    h = g - b * NH;
    c = C0 + (t & 31);
  } else if (kSpread) {
    const int u = t - kQ1 * NH * 32, lane = u & 31;
    if (lane >= NH * CR) return false;
    b = u >> 5;
    h = lane / CR;
    c = C0 + 32 + lane - h * CR;
  } else {
    const int u = t - kQ1 * NH * 32;
    b = u / (NH * CR);
    const int r = u - b * NH * CR;
    h = r / CR;
    c = C0 + 32 + r - h * CR;
  }
  yt.src = ((b * R + h * RC) * kC + c) * 2;
  yt.dst = (b * TY + h * RC) * TRow<P>::N + tpos<P>(c);
  yt.b = b;
  return true;
}

template <int P, typename Store>
__device__ __forceinline__ void y_pass(const Store* __restrict__ Sst, float2* __restrict__ Tst,
                                    const float2* __restrict__ WY, const int* __restrict__ EY,
                                    const YTask& yt) {
  using TS = TileShape<P>;
  constexpr int RC = TS::RC, RW = TS::RW;
  const Store* col = Sst + yt.src;
  float2 win[RW], dl[RW - 1];
#pragma unroll
  for (int j = 0; j < RW; ++j) win[j] = lds_pair(col + j * kC * 2);
#pragma unroll
  for (int j = 0; j < RW - 1; ++j) dl[j] = sub2(win[j + 1], win[j]);
  float2* tout = Tst + yt.dst;
  float2 W[P][P];   // tail sums of the plane's P row classes, in registers
#pragma unroll
  for (int l = 0; l < P; ++l) load_taps<P>(WY + (yt.b * P + l) * 4, W[l]);
  if (EY[yt.b])
    y_rows<P, RC, RW, true>(win, dl, W, tout);
  else
    y_rows<P, RC, RW, false>(win, dl, W, tout);
}

}  // namespace

template <int P>
struct UniformPattern {
  float wy[kQ1][P][8];                   // y taps: tail sums W_1..W_P per (b, l) at [1..P]
  float wx[kQ1][P][8];                   // x taps: tail sums W_1..W_P per (a, k) at [1..P]
  int ey[kQ1];                           // y: 1 if D(b, 0) = 0, 0 if D(b, 0) = -P
  int dx[kQ1][P];                        // x stencil start relative to the column, in [-P, 0]
};

template <int P>
struct UniformArgs {
  CUtensorMap tmap;                      // 3D map of the source state: (pair element, row, plane)
  StepArgs a;
  UniformPattern<P> pat;
  const unsigned char* std_x;            // [nx] 1 if the column follows the pattern
  const unsigned char* std_y;            // [ny]
  int gx, gy;                            // ghost columns / rows before the interior origin
};

template <int P, typename Store, bool PR>
__global__ void __launch_bounds__(TileShape<P>::NT, TileShape<P>::MINB)
    step_uniform_kernel(const __grid_constant__ UniformArgs<P> ua) {
  using TS = TileShape<P>;
  using BS = BoxShape<P, Store>;
  constexpr int TY = TS::TY, NT = TS::NT;
  constexpr int NSB = kStageBuffers;   // stage k lands in S[k % NSB], issued NSB-1 stages ahead
  constexpr int PD = NSB - 1;
  const StepArgs& a = ua.a;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_dyn + ((128 - (smem_u32(smem_dyn) & 127)) & 127);
  Store* S = reinterpret_cast<Store*>(smem_raw);                        // [NSB][box]
  float2* T = reinterpret_cast<float2*>(S + NSB * BS::STRIDE);         // [2][5][TY][TRow]
  float2* WX = T + 2 * kQ1 * TY * TRow<P>::N;                                 // [5][P][4]: (W, W)
  float2* WY = WX + kQ1 * P * 4;                                       // [5][P][4]
  int* DX = reinterpret_cast<int*>(WY + kQ1 * P * 4);                  // [5][P]
  int* EY = DX + kQ1 * P;                                              // [5]
  uint64_t* BAR = reinterpret_cast<uint64_t*>(DX + table_ints(P));    // [NSB], 8-byte aligned

  const int tid = threadIdx.x;
  const int lane = tid & 31, row = tid >> 5;
  const bool two = a.cp.npop == 2;
  const int tiles_x = (a.nx + 31) / 32;
  const int ntiles = tiles_x * ((a.ny + TY - 1) / TY);

  for (int e = tid; e < kQ1 * P * 4; e += NT) {   // tail sums, duplicated for the (f, g) lanes
    const int cl = e >> 2, al = (e & 3) + 1;
    WX[e] = bcast2((&ua.pat.wx[0][0][0])[cl * 8 + al]);
    WY[e] = bcast2((&ua.pat.wy[0][0][0])[cl * 8 + al]);
  }
  for (int e = tid; e < kQ1 * P; e += NT) (&DX[0])[e] = (&ua.pat.dx[0][0])[e];
  if (tid < kQ1) EY[tid] = ua.pat.ey[tid];
  if (tid == 0) {
    for (int k = 0; k < NSB; ++k) mbar_init(&BAR[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();  // tables and barriers

  // Global stage counter: the k-th tile of this CTA has stages 5k .. 5k+4; stage s lands in
  // S[s % NSB] and completes phase (s / NSB) & 1 of BAR[s % NSB]; it is issued PD stages ahead, so
  // the first stages of the next tile are in flight while a tile finishes and collides.
  auto issue = [&](int tile, int st, int s) {
    if (tid == 0 && tile < ntiles) {
      const int buf = (int)(s % NSB);
      const int tx0 = (tile % tiles_x) * 32, ty0 = (tile / tiles_x) * TY;
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(&BAR[buf], (unsigned)BS::BYTES);
      tma_load_3d(S + (size_t)buf * BS::STRIDE, &ua.tmap, 2 * (ua.gx + tx0 - kCO), ua.gy + ty0 - P,
                  5 * st, &BAR[buf]);
    }
  };

  YTask yt;
  const bool yon = y_task<P>(tid, yt);
#pragma unroll
  for (int k = 0; k < PD; ++k) issue(blockIdx.x, k, k);
  // Phase s (global stage counter) runs the y pass of stage s and the x pass of stage s - 1; when
  // that was the last stage of a tile, the tile collides and stores in the same phase, next to
  // the y pass of the following tile's first stage: five barriers per tile, and the FMA-heavy
  // collision of some warps overlaps the shared-memory-heavy y pass of others.
  const int my_tiles = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  int x = 0, y = 0, kx = 0;   // vertex of the tile in the x pass and its local node
  int tpo[P + 1], tpb[P + 1];
  float2 fg[kQ];      // (f, g) after streaming, velocity i = 5a + b
#pragma unroll 1
  for (int k = 0; k <= my_tiles; ++k) {
    const int tile = blockIdx.x + k * gridDim.x;   // tile of the y pass
    const bool ycur = k < my_tiles;
#pragma unroll
    for (int j = 0; j < kQ1; ++j) {
      if (!ycur && j > 0) break;   // after the last tile: its x pass of stage 4 and collision
      const int s = kQ1 * k + j;
      const bool late = ycur && !mbar_wait(&BAR[s % NSB], (unsigned)((s / NSB) & 1), a.flag);
      // stage landed (or its wait ran out: then every thread stops together, after the copies
      // still in flight -- stage s and the next stages, issued up to s + PD - 1 -- have landed)
      if (__syncthreads_or(late)) {   // also: T[(s-1)&1] written; T[s&1], S[(s+PD)%NSB] free
        // the copies in flight: stage s itself (it may still land) and the ones issued after it
        for (int t = s; t < s + PD && t < kQ1 * my_tiles; ++t)
          if (!mbar_wait(&BAR[t % NSB], (unsigned)((t / NSB) & 1), a.flag)) break;
        return;
      }
      if (ycur) {
        if (j + PD < kQ1)
          issue(tile, j + PD, s + PD);
        else
          issue(tile + gridDim.x, j + PD - kQ1, s + PD);   // the next tile's first stages
        if (yon)
          y_pass<P, Store>(S + (size_t)(s % NSB) * BS::STRIDE,
                                 T + (size_t)(s & 1) * kQ1 * TY * TRow<P>::N, WY, EY, yt);
      }
      if (k == 0 && j == 0) continue;   // no stage before the first

      // ---- x pass of stage s-1 (component st): thread = vertex; taps of (a, x mod p) ----
      const int st = (j + kQ1 - 1) % kQ1;
      if (j == 1) {   // stage 0 of tile k: this thread's vertex, its local node and stencils
        x = (tile % tiles_x) * 32 + lane;
        y = (tile / tiles_x) * TY + row;
        kx = x % P;
        // T positions of the stencil columns: the own cell (start -kx) and, for a vertex at
        // local node 0, the cell before (start -P); which one a stage takes is DX[st][kx]
#pragma unroll
        for (int al = 0; al <= P; ++al) {
          tpo[al] = tpos<P>(lane + kCO - kx + al);
          tpb[al] = tpos<P>(lane + kCO - P + al);
        }
      }
      {
        const float2* w = WX + (st * P + kx) * 4;
        const bool before = DX[st * P + kx] != -kx;   // only at kx = 0, start -P
        float2 W[P];
        load_taps<P>(w, W);
        int tp[P + 1];   // T positions of the stencil columns
#pragma unroll
        for (int al = 0; al <= P; ++al) tp[al] = before ? tpb[al] : tpo[al];
        const float2* trow0 = T + ((size_t)((s - 1) & 1) * kQ1 * TY + row) * TRow<P>::N;
#pragma unroll
        for (int b = 0; b < kQ1; ++b) {
          const float2* trow = trow0 + b * TY * TRow<P>::N;
          float2 v[P + 1];
          if constexpr (P == 2 || P == 4) {
            // even P: stencils start on a cell boundary, an even staged column, and the skew
            // moves columns by whole 16-byte units: two taps per 16-byte load
#pragma unroll
            for (int al = 0; al + 1 <= P; al += 2) {
              const float4 q = *reinterpret_cast<const float4*>(trow + tp[al]);
              v[al] = make_float2(q.x, q.y);
              v[al + 1] = make_float2(q.z, q.w);
            }
            v[P] = trow[tp[P]];
          } else {
#pragma unroll
            for (int al = 0; al <= P; ++al) v[al] = trow[tp[al]];
          }
          float2 acc = v[0];
#pragma unroll
          for (int al = 1; al <= P; ++al) acc = fma2(W[al - 1], sub2(v[al], v[al - 1]), acc);
          fg[5 * st + b] = acc;
        }
      }
      if (j != 0) continue;

      // ---- the tile of the x pass is complete: collide and store ----
      VertexMoments vm;
      const bool ok = collide_deviation_f32<PR>(fg, a.cs, a.cp, vm);
      if (x < a.nx && y < a.ny && ua.std_x[x] && ua.std_y[y]) {
        if (!ok) atomicOr(a.flag, 1);
        if (a.mom) store_moments(a.mom, a.nv, (long long)y * a.nx + x, vm);
        Store* dst = static_cast<Store*>(a.dst);
        if (!two) {   // one population: the g slots stay zero
#pragma unroll
          for (int i = 0; i < kQ; ++i) fg[i].y = 0.f;
        }
        store_images(a.ghost, x, y, [&](int xx, int yy) {
          Store* o = dst + (ptrdiff_t)yy * a.pitch + 2 * (ptrdiff_t)xx;
#pragma unroll
          for (int i = 0; i < kQ; ++i, o += a.plane_stride) st_pair(o, fg[i]);
        });
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
// SM count of a device, cached per device.
static int sm_count(int dev) {
  static std::atomic<int> cache[64];
  int n = (dev >= 0 && dev < 64) ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}
template <int P, typename Store>
static size_t smem_bytes() {
  using TS = TileShape<P>;
  using BS = BoxShape<P, Store>;
  return 128 + sizeof(Store) * kStageBuffers * BS::STRIDE + sizeof(float2) * 2 * kQ1 * TS::TY * TRow<P>::N +
         sizeof(float2) * 2 * kQ1 * P * 4 + sizeof(int) * table_ints(P) + sizeof(uint64_t) * kStageBuffers;
}

template <int P, typename Store, bool PR>
static cudaError_t launch_p(const StepArgs& a, const UniformTables& t, cudaStream_t s) {
  using TS = TileShape<P>;
  if (a.xs != 2 || a.ps != 1) return cudaErrorNotSupported;   // interleaved (f, g) pairs only
  UniformArgs<P> ua;
  memset(&ua, 0, sizeof(ua));
  ua.a = a;
  for (int c = 0; c < kQ1; ++c) {
    for (int l = 0; l < P; ++l) {
      // tail sums W_alpha = sum_{beta >= alpha} w_beta, from the FP64 weights
      for (int j = 1; j <= P; ++j) {
        double tx = 0.0, ty = 0.0;
        for (int m = j; m <= P; ++m) {
          tx += t.wx_pat[c][l][m];
          ty += t.wy_pat[c][l][m];
        }
        ua.pat.wx[c][l][j] = (float)tx;
        ua.pat.wy[c][l][j] = (float)ty;
      }
      ua.pat.dx[c][l] = t.dx_pat[c][l];
      // stencils are whole cells: D = -l, or D in {0, -P} at l = 0, on both axes (checked when
      // the tables were built; the y pass and the x-pass loads rely on it)
      if (l == 0 ? (t.dy_pat[c][0] != 0 && t.dy_pat[c][0] != -P) : t.dy_pat[c][l] != -l)
        return cudaErrorNotSupported;
      if (l == 0 ? (t.dx_pat[c][0] != 0 && t.dx_pat[c][0] != -P) : t.dx_pat[c][l] != -l)
        return cudaErrorNotSupported;
    }
    ua.pat.ey[c] = t.dy_pat[c][0] == 0 ? 1 : 0;
  }
  ua.std_x = t.std_x;
  ua.std_y = t.std_y;
  ua.gx = t.gx;
  ua.gy = t.gy;
  // tensor map over the whole source allocation (ghost cells included), pairs as 2 elements
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const char* base = static_cast<const char*>(a.src) -
                     ((ptrdiff_t)t.gy * a.pitch + 2 * (ptrdiff_t)t.gx) * (ptrdiff_t)sizeof(Store);
  const cuuint64_t dims[3] = {(cuuint64_t)a.pitch, (cuuint64_t)t.rows_alloc, (cuuint64_t)kQ};
  const cuuint64_t strides[2] = {(cuuint64_t)a.pitch * sizeof(Store),
                                 (cuuint64_t)a.plane_stride * sizeof(Store)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * kC), (cuuint32_t)TS::R, 5u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(&ua.tmap, sizeof(Store) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                   3, const_cast<char*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const size_t smem = smem_bytes<P, Store>();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  // The shared-memory opt-in is a per-device property of the kernel: set it once per device
  // (idempotent, so two threads racing on a device's first launch both set the same values).
  static std::atomic<unsigned long long> configured{0};   // per template instance, bit per device
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (!bit || !(configured.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(step_uniform_kernel<P, Store, PR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)   // all of the unified L1/shared storage as shared memory
      e = cudaFuncSetAttribute(step_uniform_kernel<P, Store, PR>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_acq_rel);
  }
  const int n_sm = sm_count(dev);
  const int ntiles = ((a.nx + 31) / 32) * ((a.ny + TS::TY - 1) / TS::TY);
  const int grid = ntiles < n_sm * TS::MINB ? ntiles : n_sm * TS::MINB;   // persistent CTAs
  step_uniform_kernel<P, Store, PR><<<grid, TS::NT, smem, s>>>(ua);
  return cudaGetLastError();
}

template <typename Store>
static cudaError_t launch_store(const StepArgs& a, const UniformTables& t, cudaStream_t s) {
  switch (a.P) {
    case 1: return a.cp.pr_on ? launch_p<1, Store, true>(a, t, s) : launch_p<1, Store, false>(a, t, s);
    case 2: return a.cp.pr_on ? launch_p<2, Store, true>(a, t, s) : launch_p<2, Store, false>(a, t, s);
    case 3: return a.cp.pr_on ? launch_p<3, Store, true>(a, t, s) : launch_p<3, Store, false>(a, t, s);
    case 4: return a.cp.pr_on ? launch_p<4, Store, true>(a, t, s) : launch_p<4, Store, false>(a, t, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step_uniform(const StepArgs& a, const UniformTables& t, int store, cudaStream_t s) {
  if (!t.valid) return cudaErrorNotSupported;
  if (store == kStoreBF16) return launch_store<__nv_bfloat16>(a, t, s);
  return launch_store<float>(a, t, s);
}

}  // namespace sllbm
