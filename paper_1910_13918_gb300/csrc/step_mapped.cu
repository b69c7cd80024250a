// Fused SLLBM step for transformed (mapped) grids, FP32 arithmetic, FP32 or BF16 deviation
// storage: pull streaming (Eq. sl_streaming) at departure points located in cell reference
// coordinates (Sec. III.E), moments, fourth-order equilibrium and BGK (Eq. streaming_fg, Pr = 1).
//
// On a mapped grid the departure cell and the local coordinates (r, s) of each (velocity, vertex)
// come from a Newton inversion of the map (precomputed once), so the interpolation does not
// separate per axis.  It stays local, though: for one velocity plane, the stencils of a tile of
// 32 x 8 neighbouring vertices fall in a small window of the source plane, displaced by about
// -xi dt.  The host computes, per tile and plane, the window's origin and the stencil origin of
// every vertex inside it (two 16-bit offsets).  The kernel copies each plane's window of (f, g)
// pairs into shared memory with one TMA tensor copy (the state layout carries ghost cells with
// the periodic images, so a window never wraps), five planes per stage, plus one copy of the
// stage's departure records (stencil origin, r, s) of the tile, two stages ahead in three
// buffers.  Every thread then interpolates its vertex from shared memory: (p+1)^2 pair loads per
// plane, weights from the local coordinates by the tail-weight polynomials, packed FP32x2
// arithmetic in the difference form of the uniform kernel (constants reproduced exactly).
// Tiles whose windows do not fit the common window size are left to the gather kernel.
#include "kernels.h"
#include "tma.cuh"

namespace sllbm {

namespace {

constexpr int kMNT = kMappedTileX * kMappedTileY;   // threads per CTA, one vertex each
constexpr int kMStages = 3;                         // staging buffers (prefetch distance 2)
constexpr int kMDesc = 3 * kQ1 * kMNT;              // 32-bit words of one stage's records

struct MappedArgs {
  CUtensorMap tmap;          // 3D map of the source state: (pair element, row, plane)
  CUtensorMap dmap;          // 4D map of the records: (column, row, plane, field)
  StepArgs a;
  const int2* org;           // [ntiles][25]: window origin (node column, node row)
  const unsigned char* tile_ok;
  int gx, gy;                // ghost columns / rows before the interior origin
  int bw, bh;                // window: bw vertices x bh rows
  int box_stride;            // Store elements between two windows in shared memory
  unsigned stage_bytes;      // bytes one stage's five copies deliver
  float wc[4][5];            // W_alpha(t) = sum_j wc[alpha-1][j] t^j, t = r - 1/2
};

// Tail weights W_1..W_P at local coordinate r (Horner in t = r - 1/2).
template <int P>
__device__ __forceinline__ void tail_weights(const float (&wc)[4][5], float r, float (&W)[P + 1]) {
  const float t = r - 0.5f;
#pragma unroll
  for (int al = 1; al <= P; ++al) {
    float acc = wc[al - 1][P];
#pragma unroll
    for (int j = P - 1; j >= 0; --j) acc = fmaf(acc, t, wc[al - 1][j]);
    W[al] = acc;
  }
}

}  // namespace

template <int P, typename Store, bool PR>
__global__ void __launch_bounds__(kMNT, 2) step_mapped_kernel(const __grid_constant__ MappedArgs ma) {
  constexpr int NSB = kMStages, PD = NSB - 1;
  const StepArgs& a = ma.a;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_dyn + ((128 - (smem_u32(smem_dyn) & 127)) & 127);
  uint32_t* D = reinterpret_cast<uint32_t*>(smem_raw);                    // [NSB][3][5][8][32]
  Store* S = reinterpret_cast<Store*>(D + (size_t)NSB * kMDesc);          // [NSB][5][box]
  uint64_t* BAR = reinterpret_cast<uint64_t*>(S + (size_t)NSB * 5 * ma.box_stride);

  const int tid = threadIdx.x;
  const int lane = tid & 31, row = tid >> 5;
  const bool two = a.cp.npop == 2;
  const int tiles_x = (a.nx + kMappedTileX - 1) / kMappedTileX;
  const int ntiles = tiles_x * ((a.ny + kMappedTileY - 1) / kMappedTileY);
  const int bw2 = 2 * ma.bw;

  float wc[4][5];
#pragma unroll
  for (int al = 0; al < 4; ++al)
#pragma unroll
    for (int j = 0; j < 5; ++j) wc[al][j] = ma.wc[al][j];

  if (tid == 0) {
    for (int k = 0; k < NSB; ++k) mbar_init(&BAR[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  // stage st of a tile = planes 5 st .. 5 st + 4, one window copy each; global stage counter as
  // in the uniform kernel
  auto issue = [&](int tile, int st, long s) {
    if (tid == 0 && tile < ntiles) {
      const int buf = (int)(s % NSB);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(&BAR[buf], ma.stage_bytes);
      tma_load_4d(D + (size_t)buf * kMDesc, &ma.dmap, (tile % tiles_x) * kMappedTileX,
                  (tile / tiles_x) * kMappedTileY, 5 * st, 0, &BAR[buf]);
      for (int b = 0; b < kQ1; ++b) {
        const int i = 5 * st + b;
        const int2 o = ma.org[(size_t)tile * kQ + i];
        tma_load_3d(S + ((size_t)buf * 5 + b) * ma.box_stride, &ma.tmap, 2 * (ma.gx + o.x), ma.gy + o.y, i,
                    &BAR[buf]);
      }
    }
  };

#pragma unroll
  for (int k = 0; k < PD; ++k) issue(blockIdx.x, k, k);
  long s0 = 0;
#pragma unroll 1
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, s0 += kQ1) {
    const int x = (tile % tiles_x) * kMappedTileX + lane, y = (tile / tiles_x) * kMappedTileY + row;
    const bool store = x < a.nx && y < a.ny && __ldg(ma.tile_ok + tile);
    float2 fg[kQ];
#pragma unroll
    for (int ph = 0; ph < kQ1; ++ph) {
      const long s = s0 + ph;
      const bool late = !mbar_wait(&BAR[s % NSB], (unsigned)((s / NSB) & 1), a.flag);   // landed
      // every thread is done with stage s - 1 (its buffer can be refilled); if the wait ran
      // out, every thread stops together after the copies in flight for the next stages
      if (__syncthreads_or(late)) {
        const long last = s0 + (long)kQ1 * ((ntiles - tile + (int)gridDim.x - 1) / (int)gridDim.x);
        for (long t = s; t < s + PD && t < last; ++t)   // stage s itself and the ones after it
          if (!mbar_wait(&BAR[t % NSB], (unsigned)((t / NSB) & 1), a.flag)) break;
        return;
      }
      if (ph + PD < kQ1)
        issue(tile, ph + PD, s + PD);
      else
        issue(tile + gridDim.x, ph + PD - kQ1, s + PD);
      const Store* stage = S + (size_t)(s % NSB) * 5 * ma.box_stride;
      const uint32_t* rec = D + (size_t)(s % NSB) * kMDesc + tid;   // [field][b][row][lane]
#pragma unroll
      for (int b = 0; b < kQ1; ++b) {
        const int lcv = (int)rec[b * kMNT];
        float Wx[P + 1], Wy[P + 1];
        tail_weights<P>(wc, __uint_as_float(rec[(kQ1 + b) * kMNT]), Wx);
        tail_weights<P>(wc, __uint_as_float(rec[(2 * kQ1 + b) * kMNT]), Wy);
        const Store* base = stage + (size_t)b * ma.box_stride + (size_t)(lcv >> 16) * bw2 + 2 * (lcv & 0xffff);
        float2 rows[P + 1];
#pragma unroll
        for (int kb = 0; kb <= P; ++kb) {
          const Store* rp = base + kb * bw2;
          float2 prev = lds_pair(rp), acc = prev;
#pragma unroll
          for (int ka = 1; ka <= P; ++ka) {
            const float2 cur = lds_pair(rp + 2 * ka);
            acc = fma2(bcast2(Wx[ka]), sub2(cur, prev), acc);
            prev = cur;
          }
          rows[kb] = acc;
        }
        float2 acc = rows[0];
#pragma unroll
        for (int kb = 1; kb <= P; ++kb) acc = fma2(bcast2(Wy[kb]), sub2(rows[kb], rows[kb - 1]), acc);
        fg[5 * ph + b] = acc;
      }
    }
    VertexMoments vm;
    const bool ok = collide_deviation_f32<PR>(fg, a.cs, a.cp, vm);
    if (store) {
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

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
template <typename Store>
static int box_stride_elems(int bw, int bh) {
  const int bytes = 2 * bw * bh * (int)sizeof(Store);
  return ((bytes + 127) / 128) * 128 / (int)sizeof(Store);
}

size_t mapped_smem_bytes(int bw, int bh, int store) {
  const int st = store == kStoreBF16 ? box_stride_elems<__nv_bfloat16>(bw, bh) * 2
                                     : box_stride_elems<float>(bw, bh) * 4;
  return 128 + (size_t)kMStages * (5 * st + 4 * kMDesc) + sizeof(uint64_t) * kMStages;
}

template <int P, typename Store, bool PR>
static cudaError_t launch_p(const StepArgs& a, const MappedTables& t, cudaStream_t s) {
  if (a.xs != 2 || a.ps != 1) return cudaErrorNotSupported;   // interleaved (f, g) pairs only
  MappedArgs ma;
  memset(&ma, 0, sizeof(ma));
  ma.a = a;
  ma.org = t.org;
  ma.tile_ok = t.tile_ok;
  ma.gx = t.gx;
  ma.gy = t.gy;
  ma.bw = t.bw;
  ma.bh = t.bh;
  ma.box_stride = box_stride_elems<Store>(t.bw, t.bh);
  ma.stage_bytes = (unsigned)(5 * 2 * t.bw * t.bh * sizeof(Store) + 4 * kMDesc);
  for (int al = 0; al < 4; ++al)
    for (int j = 0; j < 5; ++j) ma.wc[al][j] = t.wc[al][j];
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const char* base = static_cast<const char*>(a.src) -
                     ((ptrdiff_t)t.gy * a.pitch + 2 * (ptrdiff_t)t.gx) * (ptrdiff_t)sizeof(Store);
  const cuuint64_t dims[3] = {(cuuint64_t)a.pitch, (cuuint64_t)t.rows_alloc, (cuuint64_t)kQ};
  const cuuint64_t strides[2] = {(cuuint64_t)a.pitch * sizeof(Store),
                                 (cuuint64_t)a.plane_stride * sizeof(Store)};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * t.bw), (cuuint32_t)t.bh, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(&ma.tmap, sizeof(Store) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                   3, const_cast<char*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // records: [field][plane][row][column] 32-bit words, rows of dpitch columns
  const int rows = (a.ny + kMappedTileY - 1) / kMappedTileY * kMappedTileY;
  const cuuint64_t ddims[4] = {(cuuint64_t)t.dpitch, (cuuint64_t)rows, (cuuint64_t)kQ, 3u};
  const cuuint64_t dstrides[3] = {(cuuint64_t)t.dpitch * 4, (cuuint64_t)t.dpitch * rows * 4,
                                  (cuuint64_t)t.dpitch * rows * kQ * 4};
  const cuuint32_t dbox[4] = {(cuuint32_t)kMappedTileX, (cuuint32_t)kMappedTileY, 5u, 3u};
  const cuuint32_t destr[4] = {1u, 1u, 1u, 1u};
  r = enc(&ma.dmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<uint32_t*>(t.rec), ddims, dstrides,
          dbox, destr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const size_t smem = mapped_smem_bytes(t.bw, t.bh, sizeof(Store) == 2 ? kStoreBF16 : kStoreF32);
  cudaError_t e = cudaFuncSetAttribute(step_mapped_kernel<P, Store, PR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_mapped_kernel<P, Store, PR>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_mapped_kernel<P, Store, PR>, kMNT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ntiles = ((a.nx + kMappedTileX - 1) / kMappedTileX) * ((a.ny + kMappedTileY - 1) / kMappedTileY);
  const int grid = ntiles < n_sm * per_sm ? ntiles : n_sm * per_sm;   // persistent CTAs
  step_mapped_kernel<P, Store, PR><<<grid, kMNT, smem, s>>>(ma);
  return cudaGetLastError();
}

template <typename Store>
static cudaError_t launch_store(const StepArgs& a, const MappedTables& t, cudaStream_t s) {
  switch (a.P) {
    case 1: return a.cp.pr_on ? launch_p<1, Store, true>(a, t, s) : launch_p<1, Store, false>(a, t, s);
    case 2: return a.cp.pr_on ? launch_p<2, Store, true>(a, t, s) : launch_p<2, Store, false>(a, t, s);
    case 3: return a.cp.pr_on ? launch_p<3, Store, true>(a, t, s) : launch_p<3, Store, false>(a, t, s);
    case 4: return a.cp.pr_on ? launch_p<4, Store, true>(a, t, s) : launch_p<4, Store, false>(a, t, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_step_mapped(const StepArgs& a, const MappedTables& t, int store, cudaStream_t s) {
  if (!t.valid) return cudaErrorNotSupported;
  if (store == kStoreBF16) return launch_store<__nv_bfloat16>(a, t, s);
  return launch_store<float>(a, t, s);
}

}  // namespace sllbm
