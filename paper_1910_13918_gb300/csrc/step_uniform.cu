// Fused SLLBM step for uniform grids, FP32 arithmetic, FP32 or BF16 deviation storage.
//
// Pull streaming (Eq. sl_streaming) + moments + fourth-order equilibrium + BGK (Eq. streaming_fg,
// Pr = 1) in one kernel.  On a uniform grid the departure x_v - dt xi_i separates per axis and,
// away from clamped (zero-gradient) boundaries, repeats with the period p of the cells: the
// stencil offset and Lagrange weights of vertex j depend only on the velocity component and on
// the local node j mod p.  The kernel uses that "pattern":
//   * y pass: weights as a band of 2p+1 taps per (component b, local row l), passed as kernel
//     parameters and indexed with compile-time indices, applied to a register window of the
//     staged column (each staged value is read from shared memory once per column);
//   * x pass: p+1 exact taps per (component a, local column k) from shared memory.
// Vertices whose table entries differ from the pattern (next to zero-gradient boundaries) are
// not written here; the host runs the gather kernel on exactly those vertices afterwards.
//
// CTA = 32 x TY vertices (TY a multiple of p), one vertex per thread.  The 50 planes are done in
// 5 stages, one per x component a: the 10 planes (b = 0..4, f and g) of a stage are staged in
// shared memory with 16-byte cp.async copies (periodic wrap / clamp in the address), two stages
// ahead in three buffers.  Phase k runs the y pass of stage k (one thread per (plane, staged
// column), into one of two T buffers) and the x pass of stage k-1 (one thread per vertex): six
// barriers per tile.  After stage 4 every thread holds the 50
// pre-collision deviations of its vertex, collides in registers and writes 50 coalesced rows.
#include "kernels.h"

namespace sllbm {

namespace {

template <int P>
struct TileShape {
  static constexpr int TY = (P == 3) ? 15 : 16;  // multiple of p
  static constexpr int NT = 32 * TY;
  static constexpr int R = TY + 2 * P;           // staged rows y0-P .. y0+TY-1+P
  static constexpr int G = 10;                   // planes per stage
  static constexpr int BW = 2 * P + 1;           // band width
  static constexpr int BWP = (BW + 3) / 4 * 4;   // padded to float4
};

template <typename Store>
struct StoreShape {
  static constexpr int PER16 = 16 / sizeof(Store);   // elements per 16-byte chunk
  static constexpr int CO = PER16;                  // staged column origin: x0 - CO
  static constexpr int C = 32 + 2 * PER16;          // staged columns
  static constexpr int NC = C / PER16;              // chunks per staged row
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ int wrap_or_clamp(int j, int n, int periodic) {
  if (periodic) {
    j %= n;
    return j < 0 ? j + n : j;
  }
  return j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
}

}  // namespace

template <int P>
struct UniformPattern {
  float wyb[kQ1][P][TileShape<P>::BW];   // y band weights, tap j at relative row j - P
  float wx[kQ1][P][8];                   // x taps: P+1 weights, [7] unused
  int dx[kQ1][P];                        // x stencil start relative to the vertex
};

template <int P, typename Store>
struct UniformArgs {
  StepArgs a;
  UniformPattern<P> pat;
  const unsigned char* std_x;   // [nx] 1 if the column follows the pattern
  const unsigned char* std_y;   // [ny]
};

template <int P, typename Store>
__global__ void __launch_bounds__(TileShape<P>::NT, 1)
    step_uniform_kernel(const __grid_constant__ UniformArgs<P, Store> ua) {
  using TS = TileShape<P>;
  using SS = StoreShape<Store>;
  constexpr int TY = TS::TY, NT = TS::NT, R = TS::R, G = TS::G, BW = TS::BW, BWP = TS::BWP;
  constexpr int C = SS::C, NC = SS::NC, CO = SS::CO, PER16 = SS::PER16;
  constexpr int NSB = 3;   // staging buffers: stage k lands in S[k % 3], issued two phases ahead
  const StepArgs& a = ua.a;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Store* S = reinterpret_cast<Store*>(smem_raw);                       // [3][G][R][C]
  float* T = reinterpret_cast<float*>(S + NSB * G * R * C);            // [2][G][TY][C]
  float* WX = T + 2 * G * TY * C;                                     // [5][P][8]
  float* WB = WX + kQ1 * P * 8;                                       // [5][P][BWP]
  int* DX = reinterpret_cast<int*>(WB + kQ1 * P * BWP);               // [5][P]
  int* ROWOFF = DX + kQ1 * P;                                         // [R] staged row -> gy*pitch
  int* COLOFF = ROWOFF + R;                                           // [NC] chunk -> gx

  const int tid = threadIdx.x;
  const int lane = tid & 31, row = tid >> 5;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int x = x0 + lane, y = y0 + row;
  const int npop = a.cp.npop;
  const Store* src = static_cast<const Store*>(a.src);

  for (int e = tid; e < kQ1 * P * 8; e += NT) (&WX[0])[e] = (&ua.pat.wx[0][0][0])[e];
  for (int e = tid; e < kQ1 * P * BWP; e += NT) {
    const int j = e % BWP, bl = e / BWP;
    WB[e] = j < BW ? (&ua.pat.wyb[0][0][0])[bl * BW + j] : 0.f;
  }
  for (int e = tid; e < kQ1 * P; e += NT) (&DX[0])[e] = (&ua.pat.dx[0][0])[e];
  if (tid < R) ROWOFF[tid] = wrap_or_clamp(y0 - P + tid, a.ny, a.periodic_y) * a.pitch;
  if (tid >= 64 && tid < 64 + NC) {
    const int ch = tid - 64;
    int gx = x0 - CO + ch * PER16;
    if (a.periodic_x) {
      gx %= a.nx;
      if (gx < 0) gx += a.nx;
    } else {
      gx = gx < 0 ? 0 : (gx > a.pitch - PER16 ? a.pitch - PER16 : gx);
    }
    COLOFF[ch] = gx;
  }
  __syncthreads();  // tables

  // ---- staging of stage st (x component a = st): G planes x R rows x C columns ----
  auto stage_load = [&](int st) {
    constexpr int NCH = G * R * NC;
    const int buf = st % NSB;
#pragma unroll 1
    for (int e = tid; e < NCH; e += NT) {
      const int g = e / (R * NC);
      const int rem = e - g * (R * NC);
      const int r = rem / NC, ch = rem - r * NC;
      const int pop = g >= 5, b = g - 5 * pop;
      if (pop < npop) {
        const size_t plane = (size_t)(pop * kQ + 5 * st + b);
        cp_async16(S + ((size_t)(buf * G + g) * R + r) * C + ch * PER16,
                   src + plane * a.plane_stride + ROWOFF[r] + COLOFF[ch]);
      }
    }
    cp_async_commit();
  };

  stage_load(0);
  stage_load(1);

  float vals[2 * kQ];
#pragma unroll
  for (int ph = 0; ph <= kQ1; ++ph) {
    if (ph < kQ1) cp_async_wait<1>();   // stage ph landed (ph + 1 may still be in flight)
    __syncthreads();  // S[ph%3] visible; T[(ph-1)%2] written; T[ph%2] no longer read
    if (ph + 2 < kQ1)
      stage_load(ph + 2);               // its buffer held stage ph-1, consumed in phase ph-1
    else
      cp_async_commit();

    // ---- y pass of stage ph: thread = (plane g, staged column c) ----
    if (ph < kQ1 && tid < G * C) {
      const int g = tid / C, c = tid - g * C;
      const int b = g % 5;
      if (g / 5 < npop) {
        const Store* col = S + (size_t)((ph % NSB) * G + g) * R * C + c;
        float win[R];
#pragma unroll
        for (int j = 0; j < R; ++j) win[j] = to_f(col[j * C]);
        float* tout = T + ((size_t)(ph & 1) * G + g) * TY * C + c;
#pragma unroll
        for (int l = 0; l < P; ++l) {
          float wb[BWP];
          const float4* wb4 = reinterpret_cast<const float4*>(WB + (b * P + l) * BWP);
#pragma unroll
          for (int j = 0; j < BWP / 4; ++j) {
            const float4 q = wb4[j];
            wb[4 * j] = q.x;
            wb[4 * j + 1] = q.y;
            wb[4 * j + 2] = q.z;
            wb[4 * j + 3] = q.w;
          }
#pragma unroll
          for (int r = l; r < TY; r += P) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < BW; ++j) acc += wb[j] * win[r + j];
            tout[r * C] = acc;
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
    const size_t o = (size_t)y * a.pitch + x;
#pragma unroll
    for (int i = 0; i < kQ; ++i) st_store(dst + (size_t)i * a.plane_stride + o, vals[i]);
    if (npop == 2) {
#pragma unroll
      for (int i = 0; i < kQ; ++i) st_store(dst + (size_t)(kQ + i) * a.plane_stride + o, vals[kQ + i]);
    }
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
template <int P, typename Store>
static size_t smem_bytes() {
  using TS = TileShape<P>;
  using SS = StoreShape<Store>;
  return sizeof(Store) * 3 * TS::G * TS::R * SS::C + sizeof(float) * 2 * TS::G * TS::TY * SS::C +
         sizeof(float) * kQ1 * P * 8 + sizeof(float) * kQ1 * P * TS::BWP +
         sizeof(int) * (kQ1 * P + TS::R + SS::NC);
}

template <int P, typename Store>
static cudaError_t launch_p(const StepArgs& a, const UniformTables& t, cudaStream_t s) {
  using TS = TileShape<P>;
  UniformArgs<P, Store> ua;
  ua.a = a;
  for (int c = 0; c < kQ1; ++c)
    for (int l = 0; l < P; ++l) {
      for (int j = 0; j < TS::BW; ++j) ua.pat.wyb[c][l][j] = t.wy_band[c][l][j];
      for (int j = 0; j < 8; ++j) ua.pat.wx[c][l][j] = j <= P ? t.wx_pat[c][l][j] : 0.f;
      ua.pat.dx[c][l] = t.dx_pat[c][l];
    }
  ua.std_x = t.std_x;
  ua.std_y = t.std_y;
  const size_t smem = smem_bytes<P, Store>();
  static bool configured = false;  // per template instance
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(step_uniform_kernel<P, Store>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid((a.nx + 31) / 32, (a.ny + TS::TY - 1) / TS::TY);
  step_uniform_kernel<P, Store><<<grid, TS::NT, smem, s>>>(ua);
  return cudaGetLastError();
}

template <typename Store>
static cudaError_t launch_store(const StepArgs& a, const UniformTables& t, cudaStream_t s) {
  switch (a.P) {
    case 1: return launch_p<1, Store>(a, t, s);
    case 2: return launch_p<2, Store>(a, t, s);
    case 3: return launch_p<3, Store>(a, t, s);
    case 4: return launch_p<4, Store>(a, t, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step_uniform(const StepArgs& a, const UniformTables& t, int store, cudaStream_t s) {
  if (!t.valid) return cudaErrorNotSupported;
  if (store == kStoreBF16) return launch_store<__nv_bfloat16>(a, t, s);
  return launch_store<float>(a, t, s);
}

int uniform_tile_rows(int P) { return P == 3 ? 15 : 16; }

}  // namespace sllbm
