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
// Persistent CTAs (one or two per SM) walk over tiles of 32 x TY vertices (TY a multiple of p),
// one vertex per thread.  The 50 planes of a tile are done in 5 stages, one per x component a.  A stage (the 10 planes b = 0..4 of f and g) is copied into
// shared memory by two TMA tensor copies (tile + stencil halo; the state layout carries ghost
// cells with the periodic images, so a tile never wraps), completing on an mbarrier, two stages
// ahead in three buffers.  Phase k runs the y pass of stage k (task = (plane, staged column),
// register window of the column) and the x pass of stage k-1 (thread = vertex): six barriers per
// tile.  After stage 4 every thread holds the 50 pre-collision deviations of its vertex, collides
// in registers and writes 50 coalesced rows (plus periodic images in the ghost cells), while the
// first two stages of its next tile are already in flight.
#include <cuda.h>

#include "kernels.h"

namespace sllbm {

namespace {

// Tile of 32 x TY vertices; TY a multiple of p: the "tall" tile (16 rows, 15 for p = 3, one CTA
// of 512 threads per SM) or the "short" one (8 rows, 6 for p = 3, two CTAs per SM).
template <int P, bool Tall>
struct TileShape {
  static constexpr int TY = Tall ? ((P == 3) ? 15 : 16) : ((P == 3) ? 6 : 8);
  static constexpr int NT = 32 * TY;
  static constexpr int MINB = Tall ? 1 : 2;      // CTAs per SM
  static constexpr int R = TY + 2 * P;           // staged rows y0-P .. y0+TY-1+P
  static constexpr int G = 10;                   // planes per stage
};

constexpr int kStageBuffers = 3;   // TMA staging buffers per CTA (prefetch distance 2 stages)

template <typename Store>
struct StoreShape {
  static constexpr int CO = 16 / sizeof(Store);   // staged column origin x0 - CO (16-byte aligned)
  static constexpr int C = 32 + 2 * CO;           // staged columns
};

// Elements of one TMA box (5 planes x R rows x C columns), padded to 128 bytes.
template <int P, bool Tall, typename Store>
struct BoxShape {
  static constexpr int ELEMS = 5 * TileShape<P, Tall>::R * StoreShape<Store>::C;
  static constexpr int BYTES = ELEMS * (int)sizeof(Store);
  static constexpr int STRIDE = ((BYTES + 127) / 128) * 128 / (int)sizeof(Store);
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for a phase of an mbarrier with an iteration limit; on timeout set bit 2 of *flag and
// return (the results of the CTA are then garbage, but nothing hangs).
__device__ __forceinline__ void mbar_wait(uint64_t* bar, unsigned parity, int* flag) {
  for (long it = 0; it < (1L << 22); ++it)
    if (mbar_try_wait(bar, parity)) return;
  atomicOr(flag, 4);
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// y interpolation of one staged column for the rows r = l (mod p), stencil start D relative to
// the row: t[r] = sum_alpha w[alpha] * win[r + P + D + alpha]  (window row j is tile row j - P),
// evaluated as win[s] + sum_{alpha >= 1} w[alpha] (win[s + alpha] - win[s]).  Since the weights
// sum to one the two are equal, but the second reproduces a constant field exactly in FP32:
// FP32-rounded weights do not sum to one exactly, and in the first form the deficit would bias
// every uniform region the same way every step (a systematic mass drift).
template <int P, int TY, int R, int D>
__device__ __forceinline__ void y_taps(const float (&win)[R], const float (&w)[P + 1], int l,
                                       float* tout, int C) {
#pragma unroll
  for (int r = 0; r < TY; ++r) {
    if (r % P != l) continue;
    const float base = win[r + P + D];
    float acc = base;
#pragma unroll
    for (int al = 1; al <= P; ++al) acc += w[al] * (win[r + P + D + al] - base);
    tout[r * C] = acc;
  }
}

// y pass of one stage: task = (plane g, staged column c) with exact taps of (b, l).  The first
// G*32 tasks give each warp one plane (warp-uniform b, no divergence in the tap switch); the
// remaining G*(C-32) cover the right-hand staged columns.  Kept out of line: the same code
// serves the five stages of a tile, which keeps the instruction footprint small.
template <int P, int TY, int R, int G, int C, int NT, typename Store>
__device__ __noinline__ void y_pass(const Store* Sst, int box_stride, float* Tst, const float* WY,
                                    const int* DY, int npop) {
  const int tid = threadIdx.x;
#pragma unroll 1
  for (int t = tid; t < G * C; t += NT) {
    int g, c;
    if (t < G * 32) {
      g = t >> 5;
      c = t & 31;
    } else {
      g = (t - G * 32) / (C - 32);
      c = 32 + (t - G * 32) - g * (C - 32);
    }
    const int pop = g >= 5, b = g - 5 * pop;
    if (pop >= npop) continue;
    const Store* col = Sst + (size_t)pop * box_stride + (size_t)b * R * C + c;
    float win[R];
#pragma unroll
    for (int j = 0; j < R; ++j) win[j] = to_f(col[j * C]);
    float* tout = Tst + (size_t)g * TY * C + c;
#pragma unroll
    for (int l = 0; l < P; ++l) {
      float w[P + 1];
      const float* wp = WY + (b * P + l) * 8;
#pragma unroll
      for (int al = 0; al <= P; ++al) w[al] = wp[al];
      switch (DY[b * P + l]) {
        case 0: y_taps<P, TY, R, 0>(win, w, l, tout, C); break;
        case -1: y_taps<P, TY, R, -1>(win, w, l, tout, C); break;
        case -2: if constexpr (P >= 2) y_taps<P, TY, R, -2>(win, w, l, tout, C); break;
        case -3: if constexpr (P >= 3) y_taps<P, TY, R, -3>(win, w, l, tout, C); break;
        case -4: if constexpr (P >= 4) y_taps<P, TY, R, -4>(win, w, l, tout, C); break;
        default: break;
      }
    }
  }
}

}  // namespace

template <int P>
struct UniformPattern {
  float wy[kQ1][P][8];                   // y taps: P+1 weights per (b, l)
  float wx[kQ1][P][8];                   // x taps: P+1 weights per (a, k)
  int dy[kQ1][P];                        // y stencil start relative to the row, in [-P, 0]
  int dx[kQ1][P];                        // x stencil start relative to the column, in [-P, 0]
};

template <int P, typename Store>
struct UniformArgs {
  CUtensorMap tmap;                      // 3D map of the source state: (column, row, plane)
  StepArgs a;
  UniformPattern<P> pat;
  const unsigned char* std_x;            // [nx] 1 if the column follows the pattern
  const unsigned char* std_y;            // [ny]
  int gx, gy;                            // ghost columns / rows before the interior origin
};

template <int P, typename Store, bool Tall>
__global__ void __launch_bounds__(TileShape<P, Tall>::NT, TileShape<P, Tall>::MINB)
    step_uniform_kernel(const __grid_constant__ UniformArgs<P, Store> ua) {
  using TS = TileShape<P, Tall>;
  using SS = StoreShape<Store>;
  using BS = BoxShape<P, Tall, Store>;
  constexpr int TY = TS::TY, NT = TS::NT, R = TS::R, G = TS::G;
  constexpr int C = SS::C, CO = SS::CO;
  constexpr int NSB = kStageBuffers;   // stage k lands in S[k % NSB], issued NSB-1 stages ahead
  constexpr int PD = NSB - 1;
  const StepArgs& a = ua.a;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_dyn + ((128 - (smem_u32(smem_dyn) & 127)) & 127);
  Store* S = reinterpret_cast<Store*>(smem_raw);                       // [3][2][box]
  float* T = reinterpret_cast<float*>(S + NSB * 2 * BS::STRIDE);       // [2][G][TY][C]
  float* WX = T + 2 * G * TY * C;                                     // [5][P][8]
  float* WY = WX + kQ1 * P * 8;                                       // [5][P][8]
  int* DX = reinterpret_cast<int*>(WY + kQ1 * P * 8);                 // [5][P]
  int* DY = DX + kQ1 * P;                                             // [5][P]
  uint64_t* BAR = reinterpret_cast<uint64_t*>(DY + kQ1 * P);         // [NSB], 8-byte aligned

  const int tid = threadIdx.x;
  const int lane = tid & 31, row = tid >> 5;
  const int npop = a.cp.npop;
  const unsigned stage_bytes = (unsigned)(npop * BS::BYTES);
  const int tiles_x = (a.nx + 31) / 32;
  const int ntiles = tiles_x * ((a.ny + TY - 1) / TY);

  for (int e = tid; e < kQ1 * P * 8; e += NT) {
    (&WX[0])[e] = (&ua.pat.wx[0][0][0])[e];
    (&WY[0])[e] = (&ua.pat.wy[0][0][0])[e];
  }
  for (int e = tid; e < kQ1 * P; e += NT) {
    (&DX[0])[e] = (&ua.pat.dx[0][0])[e];
    (&DY[0])[e] = (&ua.pat.dy[0][0])[e];
  }
  if (tid == 0) {
    for (int k = 0; k < NSB; ++k) mbar_init(&BAR[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();  // tables and barriers

  // Global stage counter: the k-th tile of this CTA has stages 5k .. 5k+4; stage s lands in
  // S[s % 3] and completes phase (s / 3) & 1 of BAR[s % 3]; it is issued two stages ahead, so the
  // first two stages of the next tile are in flight while a tile finishes and collides.
  auto issue = [&](int tile, int st, long s) {
    if (tid == 0 && tile < ntiles) {
      const int buf = (int)(s % NSB);
      const int tx0 = (tile % tiles_x) * 32, ty0 = (tile / tiles_x) * TY;
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(&BAR[buf], stage_bytes);
      for (int pop = 0; pop < npop; ++pop)
        tma_load_3d(S + (size_t)(buf * 2 + pop) * BS::STRIDE, &ua.tmap, ua.gx + tx0 - CO,
                    ua.gy + ty0 - P, pop * kQ + 5 * st, &BAR[buf]);
    }
  };

#pragma unroll
  for (int k = 0; k < PD; ++k) issue(blockIdx.x, k, k);
  long s0 = 0;   // global index of stage 0 of the current tile
#pragma unroll 1
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, s0 += kQ1) {
    const int x0 = (tile % tiles_x) * 32, y0 = (tile / tiles_x) * TY;
    const int x = x0 + lane, y = y0 + row;
    float vals[2 * kQ];
#pragma unroll
    for (int ph = 0; ph <= kQ1; ++ph) {
      const long s = s0 + ph;
      if (ph < kQ1) mbar_wait(&BAR[s % NSB], (unsigned)((s / NSB) & 1), a.flag);  // stage landed
      __syncthreads();  // T[(s-1)&1] written; T[s&1] and S[(s+2)%3] no longer read
      if (ph + PD < kQ1)
        issue(tile, ph + PD, s + PD);
      else if (ph < kQ1)
        issue(tile + gridDim.x, ph + PD - kQ1, s + PD);   // the next tile's first stages
      if (ph < kQ1)
        y_pass<P, TY, R, G, C, NT, Store>(S + (size_t)(s % NSB) * 2 * BS::STRIDE, BS::STRIDE,
                                          T + (size_t)(s & 1) * G * TY * C, WY, DY, npop);

      // ---- x pass of stage ph-1: thread = vertex; exact taps of (a, k = x mod p) ----
      if (ph >= 1) {
        const int st = ph - 1;
        const int k = x % P;
        const float* w = WX + (st * P + k) * 8;
        const int cbase = lane + CO + DX[st * P + k];
        float wr[P + 1];
#pragma unroll
        for (int al = 0; al <= P; ++al) wr[al] = w[al];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int pop = g / 5, b = g % 5;
          const float* trow = T + (((size_t)((s - 1) & 1) * G + g) * TY + row) * C + cbase;
          const float base = trow[0];   // difference form, as in y_taps
          float acc = base;
#pragma unroll
          for (int al = 1; al <= P; ++al) acc += wr[al] * (trow[al] - base);
          vals[pop * kQ + 5 * st + b] = (pop < npop) ? acc : 0.f;
        }
      }
    }

    const bool ok = collide_deviation_f32(vals, a.cs, a.cp);
    if (x < a.nx && y < a.ny && ua.std_x[x] && ua.std_y[y]) {
      if (!ok) atomicOr(a.flag, 1);
      Store* dst = static_cast<Store*>(a.dst);
      store_images(a.ghost, x, y, [&](int xx, int yy) {
        const ptrdiff_t o = (ptrdiff_t)yy * a.pitch + xx;
#pragma unroll
        for (int i = 0; i < kQ; ++i) st_store(dst + (ptrdiff_t)i * a.plane_stride + o, vals[i]);
        if (npop == 2) {
#pragma unroll
          for (int i = 0; i < kQ; ++i)
            st_store(dst + (ptrdiff_t)(kQ + i) * a.plane_stride + o, vals[kQ + i]);
        }
      });
    }
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
template <int P, typename Store, bool Tall>
static size_t smem_bytes() {
  using TS = TileShape<P, Tall>;
  using SS = StoreShape<Store>;
  using BS = BoxShape<P, Tall, Store>;
  return 128 + sizeof(Store) * kStageBuffers * 2 * BS::STRIDE + sizeof(float) * 2 * TS::G * TS::TY * SS::C +
         sizeof(float) * 2 * kQ1 * P * 8 + sizeof(int) * (2 * kQ1 * P + 2) + sizeof(uint64_t) * kStageBuffers;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

template <int P, typename Store, bool Tall>
static cudaError_t launch_p(const StepArgs& a, const UniformTables& t, cudaStream_t s) {
  using TS = TileShape<P, Tall>;
  using SS = StoreShape<Store>;
  UniformArgs<P, Store> ua;
  memset(&ua, 0, sizeof(ua));
  ua.a = a;
  for (int c = 0; c < kQ1; ++c)
    for (int l = 0; l < P; ++l) {
      for (int j = 0; j < 8; ++j) {
        ua.pat.wx[c][l][j] = j <= P ? t.wx_pat[c][l][j] : 0.f;
        ua.pat.wy[c][l][j] = j <= P ? t.wy_pat[c][l][j] : 0.f;
      }
      ua.pat.dx[c][l] = t.dx_pat[c][l];
      ua.pat.dy[c][l] = t.dy_pat[c][l];
    }
  ua.std_x = t.std_x;
  ua.std_y = t.std_y;
  ua.gx = t.gx;
  ua.gy = t.gy;
  // tensor map over the whole source allocation (ghost cells included)
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const char* base = static_cast<const char*>(a.src) -
                     ((ptrdiff_t)t.gy * a.pitch + t.gx) * (ptrdiff_t)sizeof(Store);
  const cuuint64_t dims[3] = {(cuuint64_t)a.pitch, (cuuint64_t)t.rows_alloc, (cuuint64_t)(2 * kQ)};
  const cuuint64_t strides[2] = {(cuuint64_t)a.pitch * sizeof(Store),
                                 (cuuint64_t)a.plane_stride * sizeof(Store)};
  const cuuint32_t box[3] = {(cuuint32_t)SS::C, (cuuint32_t)TS::R, 5u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(&ua.tmap, sizeof(Store) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                   3, const_cast<char*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const size_t smem = smem_bytes<P, Store, Tall>();
  static bool configured = false;  // per template instance
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(step_uniform_kernel<P, Store, Tall>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  static int n_sm = 0;
  if (!n_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (n_sm <= 0) n_sm = 1;
  }
  const int ntiles = ((a.nx + 31) / 32) * ((a.ny + TS::TY - 1) / TS::TY);
  const int grid = ntiles < n_sm * TS::MINB ? ntiles : n_sm * TS::MINB;   // persistent CTAs
  step_uniform_kernel<P, Store, Tall><<<grid, TS::NT, smem, s>>>(ua);
  return cudaGetLastError();
}

template <typename Store, bool Tall>
static cudaError_t launch_store(const StepArgs& a, const UniformTables& t, cudaStream_t s) {
  switch (a.P) {
    case 1: return launch_p<1, Store, Tall>(a, t, s);
    case 2: return launch_p<2, Store, Tall>(a, t, s);
    case 3: return launch_p<3, Store, Tall>(a, t, s);
    case 4: return launch_p<4, Store, Tall>(a, t, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step_uniform(const StepArgs& a, const UniformTables& t, int store, cudaStream_t s) {
  if (!t.valid) return cudaErrorNotSupported;
  if (t.tall) {
    if (store == kStoreBF16) return launch_store<__nv_bfloat16, true>(a, t, s);
    return launch_store<float, true>(a, t, s);
  }
  if (store == kStoreBF16) return launch_store<__nv_bfloat16, false>(a, t, s);
  return launch_store<float, false>(a, t, s);
}

int uniform_tile_rows(int P, bool tall) {
  return tall ? (P == 3 ? 15 : 16) : (P == 3 ? 6 : 8);
}

}  // namespace sllbm
