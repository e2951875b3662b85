// NUFFT type-1 spreading (Sec. 6, step 1): b[g][f] = sum_l P[l][f] phi_x phi_y.
//
// No atomics: one CTA owns a 16 x 16-cell tile of the fine-grid window for 32
// channels; each of its 16 warps owns one tile row and each lane one channel.
// Samples are binned by (first footprint row, tile column), so the warp for
// row y reads exactly the 2w bins whose samples cover y -- first rows y-w+1..y
// in this tile column and the one to the left (a footprint of w <= 8 cells
// crosses at most one tile edge) -- and adds each sample's taps in that row to
// its private row of 16 cells in shared memory.  Every window cell is written
// exactly once, and the summation order is the sorted order, so results are
// reproducible run to run.
#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int kWarps = 16;

__global__ void __launch_bounds__(kWarps * 32) spread_kernel(const float2* __restrict__ P, int F,
                                                             const int* __restrict__ bin_start,
                                                             const int* __restrict__ sorted_l,
                                                             const int2* __restrict__ i0, const float* __restrict__ wts,
                                                             int width, int tiles, int W, float2* __restrict__ fine) {
  extern __shared__ float2 rowbuf[];  // [kWarps][kTile][32]: each warp's tile row, 32 channels
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ty = blockIdx.x / tiles, tx = blockIdx.x % tiles;
  const int f0 = blockIdx.y * 32;
  const int y = ty * kTile + warp, col0 = tx * kTile;  // this warp's window row and the tile's first column
  float2* row = rowbuf + warp * kTile * 32;
#pragma unroll
  for (int c = 0; c < kTile; ++c) row[c * 32 + lane] = make_float2(0.f, 0.f);
  const bool live = f0 + lane < F;
  const int tw = 2 * width;
  // samples whose footprint covers row y: first row in (y - w, y], tile column tx - 1 or tx
  for (int d = 0; d < width; ++d) {
    const int r0 = y - d;
    if (r0 < 0) break;
    for (int e = 0; e < 2; ++e) {
      const int tc = tx - e;
      if (tc < 0) continue;
      const int b = r0 * tiles + tc;
      const int s_end = bin_start[b + 1];
      for (int slot = bin_start[b]; slot < s_end; ++slot) {
        const int l = __ldg(sorted_l + slot);
        const int ox = __ldg(i0 + slot).x;
        const float* w = wts + (size_t)slot * tw;
        const float wy = __ldg(w + width + d);
        float2 v = live ? __ldg(P + (size_t)l * F + f0 + lane) : make_float2(0.f, 0.f);
        v.x *= wy;
        v.y *= wy;
        const int c_lo = max(0, col0 - ox), c_hi = min(width, col0 + kTile - ox);
        for (int c = c_lo; c < c_hi; ++c) {
          const float wx = __ldg(w + c);
          float2& cell = row[(ox + c - col0) * 32 + lane];
          cell.x = fmaf(v.x, wx, cell.x);
          cell.y = fmaf(v.y, wx, cell.y);
        }
      }
    }
  }
  if (live) {
    float2* dst = fine + ((size_t)y * W + col0) * F + f0 + lane;
#pragma unroll
    for (int c = 0; c < kTile; ++c) dst[(size_t)c * F] = row[c * 32 + lane];
  }
}

}  // namespace

cudaError_t launch_spread(const float2* P, int F, const int* bin_start, const int* sorted_l, const int2* i0,
                          const float* wts, int width, int tiles, int W, float2* fine, cudaStream_t s) {
  if (width > kMaxKernelWidth || W != tiles * kTile) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) * kWarps * kTile * 32;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(spread_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid(tiles * tiles, (F + 31) / 32);
  spread_kernel<<<grid, kWarps * 32, smem, s>>>(P, F, bin_start, sorted_l, i0, wts, width, tiles, W, fine);
  return cudaGetLastError();
}

}  // namespace nursd
