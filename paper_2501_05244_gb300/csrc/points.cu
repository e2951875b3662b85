// Relay-sample preparation for the NUFFT spread (Sec. 6, step 1).
//
// Each sample x_l is mapped to its fine-grid coordinate u = sigma (x - c) / delta
// (the rescaling theta = 2 pi (x - c)/(M delta) times n_f / (2 pi)), in FP64
// because |u| reaches sigma N / 2 = 256 cells and the fractional part must stay
// exact to ~1e-9.  Its footprint is the w cells i0..i0+w-1, i0 = ceil(u - w/2),
// with ES weights phi(2 (i - u) / w), phi(z) = exp(beta (sqrt(1 - z^2) - 1)).
// Samples are then sorted, stably, into 16 x 16-cell tiles of the fine-grid
// window keyed by the tile holding their first tap: a deterministic counting
// sort (per-chunk warp-level ranking with __match_any_sync, one exclusive scan
// over [bin][chunk], scatter), so the spread order -- and hence the FP32
// rounding of the result -- is reproducible run to run.
#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int kChunk = 1024;  // points per ranking warp

__global__ void points_prepare(const PointsArgs a, int2* __restrict__ i0_out, float* __restrict__ w_out,
                               int* __restrict__ bin_of, float2* __restrict__ frac_out) {
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
  bin_of[l] = (ry / kTile) * a.tiles + (rx / kTile);
}

// counts[bin][chunk] = number of points of this chunk in bin (one warp per chunk).
__global__ void points_count(const int* __restrict__ bin_of, int L, int nbins, int nchunks, int* __restrict__ counts) {
  extern __shared__ int sc[];
  const int lane = threadIdx.x;
  for (int i = lane; i < nbins; i += 32) sc[i] = 0;
  __syncwarp();
  const int base = blockIdx.x * kChunk;
  for (int it = 0; it < kChunk / 32; ++it) {
    const int l = base + it * 32 + lane;
    const int bin = (l < L) ? bin_of[l] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, bin);
    if (bin >= 0 && lane == __ffs(peers) - 1) sc[bin] += __popc(peers);
    __syncwarp();
  }
  for (int i = lane; i < nbins; i += 32) counts[(size_t)i * nchunks + blockIdx.x] = sc[i];
}

// Exclusive scan of counts (bin-major, chunk-minor) in one CTA; bin_start[b] = first slot of bin b.
__global__ void points_scan(int* __restrict__ data, int n, int nbins, int nchunks, int* __restrict__ bin_start, int L) {
  __shared__ int part[1024];
  const int tid = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int s = tid * per, e = min(n, s + per);
  int sum = 0;
  for (int i = s; i < e; ++i) sum += data[i];
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
    const int v = data[i];
    data[i] = run;
    run += v;
  }
  __syncthreads();
  for (int b = tid; b < nbins; b += 1024) bin_start[b] = data[(size_t)b * nchunks];
  if (tid == 0) bin_start[nbins] = L;
}

// Stable scatter into bin order: sorted_l, sorted i0 and sorted weights.
__global__ void points_scatter(const int* __restrict__ bin_of, const int* __restrict__ offsets, int L, int nbins,
                               int nchunks, const int2* __restrict__ i0_in, const float* __restrict__ w_in,
                               int width, int* __restrict__ sorted_l, int2* __restrict__ i0_out,
                               float* __restrict__ w_out, const float2* __restrict__ frac_in,
                               float2* __restrict__ frac_out) {
  extern __shared__ int sc[];
  const int lane = threadIdx.x;
  for (int i = lane; i < nbins; i += 32) sc[i] = 0;
  __syncwarp();
  const int base = blockIdx.x * kChunk;
  for (int it = 0; it < kChunk / 32; ++it) {
    const int l = base + it * 32 + lane;
    const int bin = (l < L) ? bin_of[l] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, bin);
    if (bin >= 0) {
      const int rank = __popc(peers & ((1u << lane) - 1u));
      const int pos = offsets[(size_t)bin * nchunks + blockIdx.x] + sc[bin] + rank;
      sorted_l[pos] = l;
      i0_out[pos] = i0_in[l];
      if (frac_out) frac_out[pos] = frac_in[l];
      for (int t = 0; t < 2 * width; ++t) w_out[(size_t)pos * 2 * width + t] = w_in[(size_t)l * 2 * width + t];
    }
    __syncwarp();
    if (bin >= 0 && lane == __ffs(peers) - 1) sc[bin] += __popc(peers);
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_points(const PointsArgs& a, int* bin_of, int2* i0_orig, float* w_orig, int* counts,
                          int* bin_start, int* sorted_l, int2* i0_sorted, float* w_sorted, cudaStream_t s,
                          float2* frac_orig, float2* frac_sorted) {
  if ((frac_orig == nullptr) != (frac_sorted == nullptr)) return cudaErrorInvalidValue;
  const int nbins = a.tiles * a.tiles;
  if (a.L <= 0) {
    cudaError_t e = cudaMemsetAsync(bin_start, 0, sizeof(int) * (nbins + 1), s);
    return e;
  }
  const int nchunks = (a.L + kChunk - 1) / kChunk;
  points_prepare<<<(a.L + 255) / 256, 256, 0, s>>>(a, i0_orig, w_orig, bin_of, frac_orig);
  const size_t smem = sizeof(int) * nbins;
  points_count<<<nchunks, 32, smem, s>>>(bin_of, a.L, nbins, nchunks, counts);
  points_scan<<<1, 1024, 0, s>>>(counts, nbins * nchunks, nbins, nchunks, bin_start, a.L);
  points_scatter<<<nchunks, 32, smem, s>>>(bin_of, counts, a.L, nbins, nchunks, i0_orig, w_orig, a.width, sorted_l,
                                          i0_sorted, w_sorted, frac_orig, frac_sorted);
  return cudaGetLastError();
}

}  // namespace nursd
