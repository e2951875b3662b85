// NUFFT type-1 spreading (Sec. 6, step 1): b[g][f] = sum_l P[l][f] phi_x phi_y.
//
// Atomic-free: one CTA owns a 16 x 16-cell tile of the fine-grid window for 32
// channels; each of its 16 warps owns one tile row and each lane one channel,
// accumulating the row's 16 cells in registers.  The samples that can touch
// the tile are those sorted into the tile's bin and the bins above / left of
// it (a footprint of w <= 8 cells crosses at most one tile edge per axis).
// They are staged in shared memory in batches (phasor row slice, 2w weights,
// footprint origin), then every warp walks the batch and adds the taps that
// fall in its row.  Each fine-grid cell is written exactly once, so the
// window needs no clearing, and the summation order is fixed by the stable
// sort.
#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int kBatch = 64;
constexpr int kWarps = kTile;  // one warp per tile row

__global__ void __launch_bounds__(kWarps * 32) spread_kernel(const float2* __restrict__ P, int F,
                                                             const int* __restrict__ bin_start,
                                                             const int* __restrict__ sorted_l,
                                                             const int2* __restrict__ i0, const float* __restrict__ wts,
                                                             int width, int tiles, int W, float2* __restrict__ fine) {
  __shared__ float2 sp[kBatch][32];
  __shared__ float sw[kBatch][2 * kMaxKernelWidth];
  __shared__ int2 si[kBatch];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ty = blockIdx.x / tiles, tx = blockIdx.x % tiles;
  const int f0 = blockIdx.y * 32;
  const int row = ty * kTile + warp;  // window row owned by this warp
  const int col0 = tx * kTile;

  // the (up to) four source bins, as a concatenated virtual list
  int rs[4], rl[4], n = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int by = ty - (k >> 1), bx = tx - (k & 1);
    int s = 0, l = 0;
    if (by >= 0 && bx >= 0) {
      const int b = by * tiles + bx;
      s = bin_start[b];
      l = bin_start[b + 1] - s;
    }
    rs[k] = s;
    rl[k] = l;
    n += l;
  }

  float2 acc[kTile];
#pragma unroll
  for (int c = 0; c < kTile; ++c) acc[c] = make_float2(0.f, 0.f);

  const int tw = 2 * width;
  for (int base = 0; base < n; base += kBatch) {
    const int nb = min(kBatch, n - base);
    __syncthreads();
    for (int idx = tid; idx < nb * 32; idx += kWarps * 32) {
      const int p = idx >> 5, c = idx & 31;
      int v = base + p, k = 0;
      while (v >= rl[k]) {
        v -= rl[k];
        ++k;
      }
      const int slot = rs[k] + v;
      const int l = __ldg(sorted_l + slot);
      sp[p][c] = (f0 + c < F) ? __ldg(P + (size_t)l * F + f0 + c) : make_float2(0.f, 0.f);
      if (c < tw) sw[p][c] = __ldg(wts + (size_t)slot * tw + c);
      if (c == 0) si[p] = __ldg(i0 + slot);
    }
    __syncthreads();
    for (int p = 0; p < nb; ++p) {
      const int2 o = si[p];
      const int dy = row - o.y;
      if ((unsigned)dy < (unsigned)width) {
        float2 v = sp[p][lane];
        const float wy = sw[p][width + dy];
        v.x *= wy;
        v.y *= wy;
        const int sh = o.x - col0;  // tap t lands in tile column sh + t
#pragma unroll
        for (int c = 0; c < kTile; ++c) {
          const int t = c - sh;
          if ((unsigned)t < (unsigned)width) {
            const float wx = sw[p][t];
            acc[c].x = fmaf(v.x, wx, acc[c].x);
            acc[c].y = fmaf(v.y, wx, acc[c].y);
          }
        }
      }
    }
  }
  if (f0 + lane < F) {
    float2* dst = fine + ((size_t)row * W + col0) * F + f0 + lane;
#pragma unroll
    for (int c = 0; c < kTile; ++c) dst[(size_t)c * F] = acc[c];
  }
}

}  // namespace

cudaError_t launch_spread(const float2* P, int F, const int* bin_start, const int* sorted_l, const int2* i0,
                          const float* wts, int width, int tiles, int W, float2* fine, cudaStream_t s) {
  if (width > kMaxKernelWidth || W != tiles * kTile) return cudaErrorInvalidValue;
  dim3 grid(tiles * tiles, (F + 31) / 32);
  spread_kernel<<<grid, kWarps * 32, 0, s>>>(P, F, bin_start, sorted_l, i0, wts, width, tiles, W, fine);
  return cudaGetLastError();
}

}  // namespace nursd
