// Relay-sample preparation for the NUFFT spread (Sec. 6, step 1).
//
// Each sample x_l is mapped to its fine-grid coordinate u = sigma (x - c) / delta
// (the rescaling theta = 2 pi (x - c)/(M delta) times n_f / (2 pi)), in FP64
// because |u| reaches sigma N / 2 = 256 cells and the fractional part must stay
// exact to ~1e-9.  Its footprint is the w cells i0..i0+w-1, i0 = ceil(u - w/2),
// with ES weights phi(2 (i - u) / w), phi(z) = exp(beta (sqrt(1 - z^2) - 1)).
// Samples are then sorted by bin = (16-cell tile column, first footprint row), tile
// column major, so the samples of one tile column over a run of rows are one
// contiguous slot range:
// counts, one exclusive scan, a scatter, an insertion sort of each (small) bin
// by sample index and a gather of the per-sample data into sorted order.  The
// order inside every bin is thus fixed, so the spread -- and the FP32 rounding
// of its sums -- is reproducible run to run.
#include "nursd_internal.cuh"

namespace nursd {
namespace {

__global__ void points_prepare(const PointsArgs a, int2* __restrict__ i0_out, float* __restrict__ w_out,
                               int* __restrict__ bin_of, float2* __restrict__ frac_out, int* __restrict__ counts) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= a.L) return;
  double dx = (double)a.xy[2 * l] - a.cx, dy = (double)a.xy[2 * l + 1] - a.cy;
  const bool ok = (fabs(dx) <= a.half_extent) && (fabs(dy) <= a.half_extent);
  if (!ok) {
    atomicOr(a.status, 1);
    dx = 0.0;
    dy = 0.0;
  }
  const double ux = dx * a.inv_fine_pitch, uy = dy * a.inv_fine_pitch;
  const double hw = 0.5 * a.width;
  const int ix = (int)ceil(ux - hw), iy = (int)ceil(uy - hw);
  float* w = w_out + (size_t)l * 2 * a.width;
  for (int t = 0; t < a.width; ++t) {
    const float zx = (float)(((double)(ix + t) - ux) / hw);
    const float zy = (float)(((double)(iy + t) - uy) / hw);
    const float px = (fabsf(zx) < 1.f) ? expf(a.beta * (sqrtf(1.f - zx * zx) - 1.f)) : 0.f;
    const float py = (fabsf(zy) < 1.f) ? expf(a.beta * (sqrtf(1.f - zy * zy) - 1.f)) : 0.f;
    w[t] = ok ? px : 0.f;
    w[a.width + t] = ok ? py : 0.f;
  }
  // The window holds every footprint of an in-range sample; the clamp only
  // guards the bin index against rounding at the aperture edge.
  const int rx = min(max(ix - a.g0, 0), a.W - 1), ry = min(max(iy - a.g0, 0), a.W - 1);
  i0_out[l] = make_int2(rx, ry);
  if (frac_out) frac_out[l] = make_float2((float)(ux - ix), (float)(uy - iy));
  const int bin = (rx / kTile) * a.W + ry;  // (tile column, footprint row)
  bin_of[l] = bin;
  atomicAdd(counts + bin, 1);
}

// Exclusive scan of the bin counts in one CTA: bin_start[b] = first sorted slot of bin b.
__global__ void points_scan(const int* __restrict__ counts, int nbins, int* __restrict__ bin_start, int L) {
  __shared__ int part[1024];
  const int tid = threadIdx.x;
  const int per = (nbins + 1023) / 1024;
  const int s = tid * per, e = min(nbins, s + per);
  int sum = 0;
  for (int i = s; i < e; ++i) sum += counts[i];
  part[tid] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = (tid >= off) ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int run = tid ? part[tid - 1] : 0;
  for (int i = s; i < e; ++i) {
    bin_start[i] = run;
    run += counts[i];
  }
  if (tid == 0) bin_start[nbins] = L;
}

__global__ void points_scatter(const int* __restrict__ bin_of, const int* __restrict__ bin_start, int L,
                               int* __restrict__ cursor, int* __restrict__ sorted_l) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= L) return;
  const int b = bin_of[l];
  sorted_l[bin_start[b] + atomicAdd(cursor + b, 1)] = l;
}

// Order each bin by sample index (insertion sort; bins hold a handful of samples), so
// the spread's summation order does not depend on the scatter's arrival order.
__global__ void points_sort_bins(const int* __restrict__ bin_start, int nbins, int* __restrict__ sorted_l) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  const int s = bin_start[b], e = bin_start[b + 1];
  for (int i = s + 1; i < e; ++i) {
    const int v = sorted_l[i];
    int j = i - 1;
    while (j >= s && sorted_l[j] > v) {
      sorted_l[j + 1] = sorted_l[j];
      --j;
    }
    sorted_l[j + 1] = v;
  }
}

__global__ void points_gather(const int* __restrict__ sorted_l, int L, int width, const int2* __restrict__ i0_in,
                              const float* __restrict__ w_in, const float2* __restrict__ frac_in,
                              int2* __restrict__ i0_out, float* __restrict__ w_out, float2* __restrict__ frac_out) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= L) return;
  const int l = sorted_l[pos];
  i0_out[pos] = i0_in[l];
  if (frac_out) frac_out[pos] = frac_in[l];
  for (int t = 0; t < 2 * width; ++t) w_out[(size_t)pos * 2 * width + t] = w_in[(size_t)l * 2 * width + t];
}

}  // namespace

int points_bins(int W, int tiles) { return W * tiles; }

cudaError_t launch_points(const PointsArgs& a, int* bin_of, int2* i0_orig, float* w_orig, int* counts,
                          int* bin_start, int* sorted_l, int2* i0_sorted, float* w_sorted, cudaStream_t s,
                          float2* frac_orig, float2* frac_sorted) {
  if ((frac_orig == nullptr) != (frac_sorted == nullptr)) return cudaErrorInvalidValue;
  const int nbins = points_bins(a.W, a.tiles);
  // counts holds 2 * nbins ints: the bin counts, then the scatter cursors
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * 2 * nbins, s);
  if (e != cudaSuccess) return e;
  if (a.L <= 0) return cudaMemsetAsync(bin_start, 0, sizeof(int) * (nbins + 1), s);
  const int blocks = (a.L + 255) / 256;
  points_prepare<<<blocks, 256, 0, s>>>(a, i0_orig, w_orig, bin_of, frac_orig, counts);
  points_scan<<<1, 1024, 0, s>>>(counts, nbins, bin_start, a.L);
  points_scatter<<<blocks, 256, 0, s>>>(bin_of, bin_start, a.L, counts + nbins, sorted_l);
  points_sort_bins<<<(nbins + 255) / 256, 256, 0, s>>>(bin_start, nbins, sorted_l);
  points_gather<<<blocks, 256, 0, s>>>(sorted_l, a.L, a.width, i0_orig, w_orig, frac_orig, i0_sorted, w_sorted,
                                      frac_sorted);
  return cudaGetLastError();
}

}  // namespace nursd
