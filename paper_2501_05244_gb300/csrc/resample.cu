// Subsampled acquisition (Methods: Sampling Criteria for NLOS, Eq. upsample2): keep every D-th relay
// sample of an N x N grid of phasors, and re-grid the kept samples to the full grid by nearest-
// neighbour or linear interpolation before a lattice reconstruction.  Both work on the temporal
// Fourier coefficients, channel-last [row][column][F] complex64.
//
// Kept sample (i, j) is grid sample (D i, D j), i, j < Nc = ceil(N / D).
//   nearest: grid index n takes kept index min(ceil(n / D - 1/2), Nc - 1) per axis (halfway: the lower);
//   linear:  between kept indices i0 = min(floor(n / D), Nc - 1) and i1 = min(i0 + 1, Nc - 1) with weight
//            t = n / D - i0 (0 past the last kept sample, which holds its value), separable in y and x.
// One thread per (row, column, channel) output, channels fastest: memory-bound streams.
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

__device__ __forceinline__ int nearest_index(int n, int D, int nc) {
  const int a = 2 * n - D;  // ceil(a / (2 D)) for a > -2D
  const int i = a <= 0 ? 0 : (a + 2 * D - 1) / (2 * D);
  return min(i, nc - 1);
}

__global__ void subsample_kernel(const float2* __restrict__ full, float2* __restrict__ kept, int N, int nc, int F,
                                 int D) {
  const long long total = (long long)nc * nc * F;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(e % F);
    const long long c = e / F;
    const int j = (int)(c % nc), i = (int)(c / nc);
    kept[e] = __ldg(full + ((size_t)(D * i) * N + (size_t)D * j) * F + f);
  }
}

__global__ void upsample_kernel(const float2* __restrict__ kept, float2* __restrict__ full, int N, int nc, int F,
                                int D, int linear) {
  const long long total = (long long)N * N * F;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(e % F);
    const long long c = e / F;
    const int x = (int)(c % N), y = (int)(c / N);
    if (!linear) {
      full[e] = __ldg(kept + ((size_t)nearest_index(y, D, nc) * nc + nearest_index(x, D, nc)) * F + f);
      continue;
    }
    const int y0 = min(y / D, nc - 1), y1 = min(y0 + 1, nc - 1);
    const int x0 = min(x / D, nc - 1), x1 = min(x0 + 1, nc - 1);
    const float ty = y1 > y0 ? (float)(y - D * y0) / (float)D : 0.f;
    const float tx = x1 > x0 ? (float)(x - D * x0) / (float)D : 0.f;
    const float2 a = __ldg(kept + ((size_t)y0 * nc + x0) * F + f), b = __ldg(kept + ((size_t)y0 * nc + x1) * F + f);
    const float2 c0 = __ldg(kept + ((size_t)y1 * nc + x0) * F + f), d = __ldg(kept + ((size_t)y1 * nc + x1) * F + f);
    // along y first (rows at x0 and x1), then along x
    const float2 r0 = make_float2((1.f - ty) * a.x + ty * c0.x, (1.f - ty) * a.y + ty * c0.y);
    const float2 r1 = make_float2((1.f - ty) * b.x + ty * d.x, (1.f - ty) * b.y + ty * d.y);
    full[e] = make_float2((1.f - tx) * r0.x + tx * r1.x, (1.f - tx) * r0.y + tx * r1.y);
  }
}

unsigned grid_for(long long total) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long want = (total + 255) / 256;
  return (unsigned)std::max<long long>(1, std::min<long long>(want, 16LL * sms));
}

}  // namespace

cudaError_t launch_subsample(const float2* full, float2* kept, int N, int F, int D, cudaStream_t s) {
  const int nc = (N + D - 1) / D;
  const long long total = (long long)nc * nc * F;
  subsample_kernel<<<grid_for(total), 256, 0, s>>>(full, kept, N, nc, F, D);
  return cudaGetLastError();
}

cudaError_t launch_upsample(const float2* kept, float2* full, int N, int F, int D, int linear, cudaStream_t s) {
  const int nc = (N + D - 1) / D;
  const long long total = (long long)N * N * F;
  upsample_kernel<<<grid_for(total), 256, 0, s>>>(kept, full, N, nc, F, D, linear);
  return cudaGetLastError();
}

}  // namespace nursd
