// NUFFT type-1 spreading (Sec. 6, step 1): b[g][f] = sum_l P[l][f] phi_x phi_y.
//
// No atomics: one CTA owns a 16 x 16-cell tile of the fine-grid window for 32
// channels; each of its 16 warps owns one tile row, each lane one channel, and
// the row's 16 cells live in registers.  Samples are binned by (tile column,
// first footprint row), tile column major, so the samples that can touch the
// tile -- first rows ty*16-w+1 .. ty*16+15 in this tile column and the one to
// its left (a footprint of w <= 8 cells crosses at most one tile edge) -- are
// two contiguous slot ranges.  The CTA stages them in shared memory (the 32
// channels of each sample's phasor, its footprint origin and its x and y
// weights) in chunks -- one round of loads when P is already in sorted-slot order,
// two when its rows are found through the sorted index -- and the warp for row y
// adds the samples whose first row is in y-w+1 .. y (again two contiguous sub-ranges).  A sample's taps land on cells
// o .. o+w-1 of the row, o = its first column minus the tile's; a warp-uniform
// switch on o selects a fully unrolled update of the registers it touches.
// Every window cell is written exactly once, and the summation order is the
// sorted order, so results are reproducible run to run.
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int kWarps = kTile;  // one warp per tile row
constexpr int kCh = 32;        // channels per CTA
constexpr int kCap = 256;      // samples staged per chunk

struct SpreadSmem {
  float2 p[kCap][kCh];   // phasor slices
  float wx[kCap][8];     // x weights (first w used)
  float wy[kCap][8];     // y weights
  float wt[kCap][kTile]; // y weight of each row of the tile (0 where the footprint misses it)
  int o[kCap];           // first footprint column relative to the tile's
  int oy[kCap];          // first footprint row relative to the tile's
  int l[kCap];           // sample index (row of P)
};

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 8 : 0) : "memory");
}

// acc[O + c] += v * wx[c] for the taps c < KW that fall inside the row (O is a constant).
template <int KW, int O>
__device__ __forceinline__ void add_taps(float2 (&acc)[kTile], float2 v, const float (&wx)[8]) {
#pragma unroll
  for (int c = 0; c < KW; ++c) {
    if (O + c >= 0 && O + c < kTile) {
      acc[O + c].x = fmaf(v.x, wx[c], acc[O + c].x);
      acc[O + c].y = fmaf(v.y, wx[c], acc[O + c].y);
    }
  }
}

template <int KW>
__device__ __forceinline__ void add_sample(float2 (&acc)[kTile], int o, float2 v, const float (&wx)[8]) {
  switch (o) {
#define NURSD_TAP_CASE(O) \
  case O:                 \
    add_taps<KW, O>(acc, v, wx); \
    break;
    NURSD_TAP_CASE(-7) NURSD_TAP_CASE(-6) NURSD_TAP_CASE(-5) NURSD_TAP_CASE(-4) NURSD_TAP_CASE(-3)
    NURSD_TAP_CASE(-2) NURSD_TAP_CASE(-1) NURSD_TAP_CASE(0) NURSD_TAP_CASE(1) NURSD_TAP_CASE(2)
    NURSD_TAP_CASE(3) NURSD_TAP_CASE(4) NURSD_TAP_CASE(5) NURSD_TAP_CASE(6) NURSD_TAP_CASE(7)
    NURSD_TAP_CASE(8) NURSD_TAP_CASE(9) NURSD_TAP_CASE(10) NURSD_TAP_CASE(11) NURSD_TAP_CASE(12)
    NURSD_TAP_CASE(13) NURSD_TAP_CASE(14) NURSD_TAP_CASE(15)
#undef NURSD_TAP_CASE
    default:
      break;  // the footprint ends left of the tile
  }
}

template <int KW>
__global__ void __launch_bounds__(kWarps * 32, 2) spread_kernel(const float2* __restrict__ P, int F,
                                                                const int* __restrict__ bin_start,
                                                                const int* __restrict__ sorted_l,
                                                                const int2* __restrict__ i0,
                                                                const float* __restrict__ wts, int tiles, int W,
                                                                float2* __restrict__ fine) {
  extern __shared__ __align__(16) unsigned char raw[];
  SpreadSmem& sm = *reinterpret_cast<SpreadSmem*>(raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ty = blockIdx.x / tiles, tx = blockIdx.x % tiles;
  const int f0 = blockIdx.y * kCh;
  const int y = ty * kTile + warp, col0 = tx * kTile;
  // slot ranges of the two tile columns over first rows rlo .. rhi (bin = column * W + row)
  const int rlo = max(ty * kTile - KW + 1, 0), rhi1 = ty * kTile + kTile;
  const int aS = tx > 0 ? bin_start[(tx - 1) * W + rlo] : 0;
  const int nA = tx > 0 ? bin_start[(tx - 1) * W + rhi1] - aS : 0;
  const int bS = bin_start[tx * W + rlo];
  const int n = nA + bin_start[tx * W + rhi1] - bS;
  // this warp's samples (first rows wlo .. y), as indices into the concatenated ranges
  const int wlo = max(y - KW + 1, 0);
  const int wa0 = tx > 0 ? bin_start[(tx - 1) * W + wlo] - aS : 0;
  const int wa1 = tx > 0 ? bin_start[(tx - 1) * W + y + 1] - aS : 0;
  const int wb0 = nA + bin_start[tx * W + wlo] - bS;
  const int wb1 = nA + bin_start[tx * W + y + 1] - bS;

  float2 acc[kTile];
#pragma unroll
  for (int c = 0; c < kTile; ++c) acc[c] = make_float2(0.f, 0.f);
  const bool live = f0 + lane < F;
  for (int c0 = 0; c0 < n; c0 += kCap) {
    const int cn = min(kCap, n - c0);
    __syncthreads();  // the previous chunk has been consumed
    // phase 1, one thread per sample (all loads in flight at once): index, origin, weights; when P
    // is in slot order its copies need no index and start here too
    if (!sorted_l)
      for (int s = warp; s < cn; s += kWarps) {
        const int v = c0 + s;
        const int slot = v < nA ? aS + v : bS + (v - nA);
        cp_async8(&sm.p[s][lane], live ? P + (size_t)slot * F + f0 + lane : P, live);
      }
    for (int s = threadIdx.x; s < cn; s += kWarps * 32) {
      const int v = c0 + s;
      const int slot = v < nA ? aS + v : bS + (v - nA);
      const int l = sorted_l ? __ldg(sorted_l + slot) : slot;
      const int2 o = __ldg(i0 + slot);
      const float* w = wts + (size_t)slot * 2 * KW;
      float wv[2 * KW];
#pragma unroll
      for (int t = 0; t < 2 * KW; ++t) wv[t] = __ldg(w + t);
      sm.l[s] = l;
      sm.o[s] = o.x - col0;
      sm.oy[s] = o.y - ty * kTile;
#pragma unroll
      for (int t = 0; t < KW; ++t) {
        sm.wx[s][t] = wv[t];
        sm.wy[s][t] = wv[KW + t];
      }
    }
    __syncthreads();
    // phase 2, one warp per sample: its 32 channels of P (sample order), and its y weight for each tile row
    for (int s = warp; s < cn; s += kWarps) {
      if (sorted_l) cp_async8(&sm.p[s][lane], live ? P + (size_t)sm.l[s] * F + f0 + lane : P, live);
      if (lane < kTile) {
        const int d = lane - sm.oy[s];
        sm.wt[s][lane] = (d >= 0 && d < KW) ? sm.wy[s][d] : 0.f;
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int c1 = c0 + cn;
    auto visit = [&](int s) {
      const float wyv = sm.wt[s][warp];
      float2 pv = sm.p[s][lane];
      pv.x *= wyv;
      pv.y *= wyv;
      float wx[8];
      const float4 w0 = *reinterpret_cast<const float4*>(&sm.wx[s][0]);
      const float4 w1 = *reinterpret_cast<const float4*>(&sm.wx[s][4]);
      wx[0] = w0.x; wx[1] = w0.y; wx[2] = w0.z; wx[3] = w0.w;
      wx[4] = w1.x; wx[5] = w1.y; wx[6] = w1.z; wx[7] = w1.w;
      add_sample<KW>(acc, sm.o[s], pv, wx);
    };
    {  // left tile column: only samples whose footprint reaches this tile
      const int s1 = min(wa1, c1) - c0;
      for (int s = max(wa0, c0) - c0; s < s1; ++s)
        if (sm.o[s] > -KW) visit(s);
    }
    {  // this tile column
      const int s1 = min(wb1, c1) - c0;
      for (int s = max(wb0, c0) - c0; s < s1; ++s) visit(s);
    }
  }
  if (live) {
    float2* dst = fine + ((size_t)y * W + col0) * F + f0 + lane;
#pragma unroll
    for (int c = 0; c < kTile; ++c) dst[(size_t)c * F] = acc[c];
  }
}

template <int KW>
cudaError_t launch_kw(const float2* P, int F, const int* bin_start, const int* sorted_l, const int2* i0,
                      const float* wts, int tiles, int W, float2* fine, cudaStream_t s) {
  const size_t smem = sizeof(SpreadSmem);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(spread_kernel<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid(tiles * tiles, (F + kCh - 1) / kCh);
  spread_kernel<KW><<<grid, kWarps * 32, smem, s>>>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_spread(const float2* P, int F, const int* bin_start, const int* sorted_l, const int2* i0,
                          const float* wts, int width, int tiles, int W, float2* fine, cudaStream_t s) {
  if (W != tiles * kTile) return cudaErrorInvalidValue;
  switch (width) {
    case 4: return launch_kw<4>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, s);
    case 5: return launch_kw<5>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, s);
    case 6: return launch_kw<6>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, s);
    case 7: return launch_kw<7>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, s);
    case 8: return launch_kw<8>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nursd
