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
// CTA = 32 x TY vertices (TY a multiple of p), one vertex per thread.  The 50 planes are done in
// 5 stages, one per x component a.  A stage (the 10 planes b = 0..4 of f and g) is copied into
// shared memory by two TMA tensor copies (tile + stencil halo; the state layout carries ghost
// cells with the periodic images, so a tile never wraps), completing on an mbarrier, two stages
// ahead in three buffers.  Phase k runs the y pass of stage k (task = (plane, staged column),
// register window of the column) and the x pass of stage k-1 (thread = vertex): six barriers per
// tile.  After stage 4 every thread holds the 50 pre-collision deviations of its vertex, collides
// in registers and writes 50 coalesced rows (plus periodic images in the ghost cells).
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
// the row: t[r] = sum_alpha w[alpha] * win[r + P + D + alpha]  (window row j is tile row j - P).
template <int P, int TY, int R, int D>
__device__ __forceinline__ void y_taps(const float (&win)[R], const float (&w)[P + 1], int l,
                                       float* tout, int C) {
#pragma unroll
  for (int r = 0; r < TY; ++r) {
    if (r % P != l) continue;
    float acc = 0.f;
#pragma unroll
    for (int al = 0; al <= P; ++al) acc += w[al] * win[r + P + D + al];
    tout[r * C] = acc;
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
  constexpr int NSB = 3;   // staging buffers: stage k lands in S[k % 3], issued two phases ahead
  const StepArgs& a = ua.a;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_dyn + ((128 - (smem_u32(smem_dyn) & 127)) & 127);
  Store* S = reinterpret_cast<Store*>(smem_raw);                       // [3][2][box]
  float* T = reinterpret_cast<float*>(S + NSB * 2 * BS::STRIDE);       // [2][G][TY][C]
  float* WX = T + 2 * G * TY * C;                                     // [5][P][8]
  float* WY = WX + kQ1 * P * 8;                                       // [5][P][8]
  int* DX = reinterpret_cast<int*>(WY + kQ1 * P * 8);                 // [5][P]
  int* DY = DX + kQ1 * P;                                             // [5][P]
  uint64_t* BAR = reinterpret_cast<uint64_t*>(DY + kQ1 * P);         // [3], 8-byte aligned

  const int tid = threadIdx.x;
  const int lane = tid & 31, row = tid >> 5;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int x = x0 + lane, y = y0 + row;
  const int npop = a.cp.npop;
  const unsigned stage_bytes = (unsigned)(npop * BS::BYTES);

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

  // ---- stage st (x component a = st): two TMA boxes (f, g) of 5 planes x R rows x C cols ----
  auto stage_load = [&](int st) {
    if (tid == 0) {
      const int buf = st % NSB;
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(&BAR[buf], stage_bytes);
      const int cx = ua.gx + x0 - CO, cy = ua.gy + y0 - P;
      for (int pop = 0; pop < npop; ++pop)
        tma_load_3d(S + (size_t)(buf * 2 + pop) * BS::STRIDE, &ua.tmap, cx, cy, pop * kQ + 5 * st,
                    &BAR[buf]);
    }
  };

  stage_load(0);
  stage_load(1);

  float vals[2 * kQ];
#pragma unroll
  for (int ph = 0; ph <= kQ1; ++ph) {
    if (ph < kQ1) mbar_wait(&BAR[ph % NSB], (ph / NSB) & 1, a.flag);   // stage ph landed
    __syncthreads();  // T[(ph-1)%2] written; T[ph%2] and S[(ph+2)%3] no longer read
    if (ph + 2 < kQ1) stage_load(ph + 2);   // its buffer held stage ph-1, consumed in phase ph-1

    // ---- y pass of stage ph: task = (plane g, staged column c), exact taps of (b, l) ----
    if (ph < kQ1) {
#pragma unroll 1
      for (int t = tid; t < G * C; t += NT) {
        // the first G*32 tasks give each warp one plane (warp-uniform b, no divergence in the
        // tap switch); the remaining G*(C-32) cover the right-hand staged columns
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
        const Store* col = S + (size_t)((ph % NSB) * 2 + pop) * BS::STRIDE + (size_t)b * R * C + c;
        float win[R];
#pragma unroll
        for (int j = 0; j < R; ++j) win[j] = to_f(col[j * C]);
        float* tout = T + ((size_t)(ph & 1) * G + g) * TY * C + c;
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
        const float* trow = T + (((size_t)(st & 1) * G + g) * TY + row) * C + cbase;
        float acc = 0.f;
#pragma unroll
        for (int al = 0; al <= P; ++al) acc += wr[al] * trow[al];
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

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
template <int P, typename Store, bool Tall>
static size_t smem_bytes() {
  using TS = TileShape<P, Tall>;
  using SS = StoreShape<Store>;
  using BS = BoxShape<P, Tall, Store>;
  return 128 + sizeof(Store) * 3 * 2 * BS::STRIDE + sizeof(float) * 2 * TS::G * TS::TY * SS::C +
         sizeof(float) * 2 * kQ1 * P * 8 + sizeof(int) * (2 * kQ1 * P + 2) + sizeof(uint64_t) * 3;
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
  dim3 grid((a.nx + 31) / 32, (a.ny + TS::TY - 1) / TS::TY);
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
