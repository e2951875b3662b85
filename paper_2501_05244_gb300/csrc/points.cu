// Relay-sample preparation for the NUFFT spread (Sec. 6, step 1).
//
// Each sample x_l is mapped to its fine-grid coordinate u = sigma (x - c) / delta
// (the rescaling theta = 2 pi (x - c)/(M delta) times n_f / (2 pi)), in FP64
// because |u| reaches sigma N / 2 = 256 cells and the fractional part must stay
// exact to ~1e-9.  Its footprint is the w cells i0..i0+w-1, i0 = ceil(u - w/2),
// with ES weights phi(2 (i - u) / w), phi(z) = exp(beta (sqrt(1 - z^2) - 1)).
// Samples are then sorted by bin = (16-cell tile column, edge flag, first footprint
// row), where the edge flag marks footprints that cross into the next tile column,
// so the samples of one tile column (and of its edge part) over a run of rows are
// one contiguous slot range:
// counts, one exclusive scan, a scatter, an insertion sort of each (small) bin
// by sample index and a gather of the per-sample data into sorted order.  The
// order inside every bin is thus fixed, so the spread -- and the FP32 rounding
// of its sums -- is reproducible run to run.
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

// The samples of one call (OneItem) or of the items of a batched call (PointsItems, item = blockIdx.y,
// its per-sample arrays at item * pts, its counts at item * cstride and its bin_start at item * bstride).
struct OneItem {
  int L;
  const float* xy;
  __device__ int len(int) const { return L; }
  __device__ const float* pos(int) const { return xy; }
};
struct ManyItems {
  PointsItems it;
  __device__ int len(int b) const { return it.L[b]; }
  __device__ const float* pos(int b) const { return it.xy[b]; }
};
struct Strides {
  long long pts;  // per-sample arrays
  int cstride;    // counts and cursors (2 nbins)
  int bstride;    // bin_start (nbins + 1)
};

template <class Src>
__global__ void points_prepare(const PointsArgs a, const Src src, const Strides st, int2* __restrict__ i0_out,
                               float* __restrict__ w_out, int* __restrict__ bin_of, float2* __restrict__ frac_out,
                               int* __restrict__ counts) {
  const int item = blockIdx.y;
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= src.len(item)) return;
  const float* xy = src.pos(item);
  const long long po = item * st.pts;
  i0_out += po;
  w_out += po * 2 * a.width;
  bin_of += po;
  if (frac_out) frac_out += po;
  counts += (size_t)item * st.cstride;
  double dx = (double)xy[2 * l] - a.cx, dy = (double)xy[2 * l + 1] - a.cy;
  const bool ok = (fabs(dx) <= a.half_extent) && (fabs(dy) <= a.half_extent);
  if (!ok) {
    atomicOr(a.status, 1);
    dx = 0.0;
    dy = 0.0;
  }
  const double ux = dx * a.inv_fine_pitch, uy = dy * a.inv_fine_pitch;
  const double hw = 0.5 * a.width;
  const int ix = (int)ceil(ux - hw), iy = (int)ceil(uy - hw);
  // tap t sits at z = (i0 + t - u) / (w / 2): the offset i0 - u in (-w/2 - 1, -w/2] is exact
  // enough in fp32 once taken in fp64, so the taps need no fp64 division
  const float fx = (float)((double)ix - ux), fy = (float)((double)iy - uy);
  const float inv_hw = 2.f / (float)a.width;
  float* w = w_out + (size_t)l * 2 * a.width;
  for (int t = 0; t < a.width; ++t) {
    const float zx = (fx + (float)t) * inv_hw;
    const float zy = (fy + (float)t) * inv_hw;
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
  // (tile column, whether the footprint crosses into the next tile column, footprint row)
  const int edge = (rx % kTile) + a.width > kTile ? 1 : 0;
  const int bin = ((rx / kTile) * 2 + edge) * a.W + ry;
  bin_of[l] = bin;
  atomicAdd(counts + bin, 1);
}

// Exclusive scan of the bin counts in one CTA: bin_start[b] = first sorted slot of bin b.
// The counts are staged in shared memory with coalesced loads (kScanChunk at a time, all of a
// chunk's loads in flight at once), each thread scans a contiguous run of `per` counts (runs
// padded by one word, so the threads of a warp hit distinct banks), and the runs' totals are
// scanned with warp shuffles.  1024 threads and a 36,864-count chunk (148 KB): the 34,848 bins of
// a 528-cell window in one pass (nine 4,096-count passes took 30 us, each waiting on its loads).
constexpr int kScanThreads = 1024, kScanChunk = 36864;
constexpr size_t kScanSmem = sizeof(int) * (size_t)kScanThreads * (kScanChunk / kScanThreads + 1);
static_assert(kScanThreads % 32 == 0 && kScanThreads <= 1024 && kScanChunk % kScanThreads == 0, "scan shape");
// One CTA per item (blockIdx.x).
template <class Src>
__global__ void __launch_bounds__(kScanThreads) points_scan(const int* __restrict__ counts, int nbins,
                                                           int* __restrict__ bin_start, const Src src,
                                                           const Strides st) {
  constexpr int per = kScanChunk / kScanThreads, nw = kScanThreads / 32;
  const int L = src.len(blockIdx.x);
  counts += (size_t)blockIdx.x * st.cstride;
  bin_start += (size_t)blockIdx.x * st.bstride;
  extern __shared__ int buf[];  // kScanThreads runs of per + 1 words
  __shared__ int warp_sum[nw];
  __shared__ int carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto slot = [](int i) { return (i / per) * (per + 1) + i % per; };  // padded position of count i
  if (tid == 0) carry = 0;
  for (int c0 = 0; c0 < nbins; c0 += kScanChunk) {
    const int cn = min(kScanChunk, nbins - c0);
    // every count of the chunk copied at once (past cn: zero-filled)
#pragma unroll
    for (int k = 0; k < per; ++k) {
      const int i = tid + k * kScanThreads;
      const unsigned d = (unsigned)__cvta_generic_to_shared(buf + slot(i));
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(counts + (i < cn ? c0 + i : 0)),
                   "r"(i < cn ? 4 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    int* run_p = buf + tid * (per + 1);
    int run = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) run += run_p[k];
    int incl = run;  // inclusive scan of the runs within the warp
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    if (warp == 0) {  // scan of the nw warp totals (lanes beyond them carry zeros)
      const int ws = lane < nw ? warp_sum[lane] : 0;
      int wincl = ws;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, wincl, off);
        if (lane >= off) wincl += v;
      }
      if (lane < nw) warp_sum[lane] = wincl - ws;  // exclusive
    }
    __syncthreads();
    int pos = carry + warp_sum[warp] + incl - run;
    const int total = carry + warp_sum[nw - 1] + __shfl_sync(0xffffffffu, incl, 31);
#pragma unroll
    for (int k = 0; k < per; ++k) {
      const int v = run_p[k];
      run_p[k] = pos;
      pos += v;
    }
    __syncthreads();
    for (int i = tid; i < cn; i += kScanThreads) bin_start[c0 + i] = buf[slot(i)];
    if (tid == kScanThreads - 1) carry = total;
    __syncthreads();
  }
  if (tid == 0) bin_start[nbins] = L;
}

template <class Src>
__global__ void points_scatter(const int* __restrict__ bin_of, const int* __restrict__ bin_start, const Src src,
                               const Strides st, int* __restrict__ cursor, int* __restrict__ sorted_l,
                               int nbins, int* __restrict__ status) {
  const int item = blockIdx.y;
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= src.len(item)) return;
  bin_of += item * st.pts;
  sorted_l += item * st.pts;
  bin_start += (size_t)item * st.bstride;
  cursor += (size_t)item * st.cstride;
  const int b = bin_of[l];
  if (!NURSD_CHECK(b >= 0 && b < nbins, status)) return;
  const int slot = bin_start[b] + atomicAdd(cursor + b, 1);
  if (NURSD_CHECK(slot >= 0 && slot < src.len(item), status)) sorted_l[slot] = l;
}

// Order each bin by sample index (insertion sort; bins hold a handful of samples), so
// the spread's summation order does not depend on the scatter's arrival order.  Bins of
// up to kSortLocal samples are sorted in a thread-local array, larger ones in place.
constexpr int kSortLocal = 32;
__global__ void points_sort_bins(const int* __restrict__ bin_start, int nbins, int* __restrict__ sorted_l,
                                 const Strides st) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  bin_start += (size_t)blockIdx.y * st.bstride;
  sorted_l += blockIdx.y * st.pts;
  const int s = bin_start[b], e = bin_start[b + 1];
  if (e - s <= kSortLocal) {
    int v[kSortLocal];
    const int k = e - s;
    for (int i = 0; i < k; ++i) v[i] = sorted_l[s + i];
    for (int i = 1; i < k; ++i) {
      const int x = v[i];
      int j = i - 1;
      while (j >= 0 && v[j] > x) {
        v[j + 1] = v[j];
        --j;
      }
      v[j + 1] = x;
    }
    for (int i = 0; i < k; ++i) sorted_l[s + i] = v[i];
    return;
  }
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

template <class Src>
__global__ void points_gather(const int* __restrict__ sorted_l, const Src src, const Strides st, int width,
                              const int2* __restrict__ i0_in, const float* __restrict__ w_in,
                              const float2* __restrict__ frac_in, int2* __restrict__ i0_out,
                              float* __restrict__ w_out, float2* __restrict__ frac_out, int* __restrict__ slot_of,
                              int* __restrict__ status) {
  const int item = blockIdx.y;
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= src.len(item)) return;
  const long long po = item * st.pts;
  sorted_l += po;
  i0_in += po;
  i0_out += po;
  w_in += po * 2 * width;
  w_out += po * 2 * width;
  if (frac_in) frac_in += po;
  if (frac_out) frac_out += po;
  if (slot_of) slot_of += po;
  const int l = sorted_l[pos];
  if (!NURSD_CHECK(l >= 0 && l < src.len(item), status)) return;
  if (slot_of) slot_of[l] = pos;
  i0_out[pos] = i0_in[l];
  if (frac_out) frac_out[pos] = frac_in[l];
  for (int t = 0; t < 2 * width; ++t) w_out[(size_t)pos * 2 * width + t] = w_in[(size_t)l * 2 * width + t];
}

}  // namespace

int points_bins(int W, int tiles) { return 2 * W * tiles; }

namespace {
template <class Src>
cudaError_t launch_points_on(const PointsArgs& a, const Src& src, int n, int maxL, const Strides& st, int* bin_of,
                             int2* i0_orig, float* w_orig, int* counts, int* bin_start, int* sorted_l,
                             int2* i0_sorted, float* w_sorted, cudaStream_t s, float2* frac_orig, float2* frac_sorted,
                             int* slot_of) {
  const int nbins = points_bins(a.W, a.tiles);
  const dim3 grid((unsigned)std::max(1, (maxL + 255) / 256), (unsigned)n);
  points_prepare<<<grid, 256, 0, s>>>(a, src, st, i0_orig, w_orig, bin_of, frac_orig, counts);
  static bool scan_configured = false;  // per Src instantiation
  if (!scan_configured) {
    const cudaError_t e =
        cudaFuncSetAttribute(points_scan<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScanSmem);
    if (e != cudaSuccess) return e;
    scan_configured = true;
  }
  points_scan<<<n, kScanThreads, kScanSmem, s>>>(counts, nbins, bin_start, src, st);
  points_scatter<<<grid, 256, 0, s>>>(bin_of, bin_start, src, st, counts + nbins, sorted_l, nbins, a.status);
  points_sort_bins<<<dim3((nbins + 255) / 256, (unsigned)n), 256, 0, s>>>(bin_start, nbins, sorted_l, st);
  points_gather<<<grid, 256, 0, s>>>(sorted_l, src, st, a.width, i0_orig, w_orig, frac_orig, i0_sorted, w_sorted,
                                     frac_sorted, slot_of, a.status);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_points(const PointsArgs& a, int* bin_of, int2* i0_orig, float* w_orig, int* counts,
                          int* bin_start, int* sorted_l, int2* i0_sorted, float* w_sorted, cudaStream_t s,
                          float2* frac_orig, float2* frac_sorted, int* slot_of) {
  if ((frac_orig == nullptr) != (frac_sorted == nullptr)) return cudaErrorInvalidValue;
  const int nbins = points_bins(a.W, a.tiles);
  // counts holds 2 * nbins ints: the bin counts, then the scatter cursors
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * 2 * nbins, s);
  if (e != cudaSuccess) return e;
  if (a.L <= 0) return cudaMemsetAsync(bin_start, 0, sizeof(int) * (nbins + 1), s);
  return launch_points_on(a, OneItem{a.L, a.xy}, 1, a.L, Strides{0, 0, 0}, bin_of, i0_orig, w_orig, counts,
                          bin_start, sorted_l, i0_sorted, w_sorted, s, frac_orig, frac_sorted, slot_of);
}

cudaError_t launch_points_batched(const PointsArgs& a, const PointsItems& items, int n, long long pts, int* bin_of,
                                  int2* i0_orig, float* w_orig, int* counts, int* bin_start, int* sorted_l,
                                  int2* i0_sorted, float* w_sorted, float2* frac_orig, float2* frac_sorted,
                                  int* slot_of, cudaStream_t s) {
  if (n < 1 || n > kMaxBatch || (frac_orig == nullptr) != (frac_sorted == nullptr)) return cudaErrorInvalidValue;
  const int nbins = points_bins(a.W, a.tiles);
  int maxL = 0;
  for (int b = 0; b < n; ++b) {
    if (items.L[b] < 0 || items.L[b] > pts) return cudaErrorInvalidValue;
    maxL = std::max(maxL, items.L[b]);
  }
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * 2 * nbins * (size_t)n, s);
  if (e != cudaSuccess) return e;
  return launch_points_on(a, ManyItems{items}, n, maxL, Strides{pts, 2 * nbins, nbins + 1}, bin_of, i0_orig, w_orig,
                          counts, bin_start, sorted_l, i0_sorted, w_sorted, s, frac_orig, frac_sorted, slot_of);
}

}  // namespace nursd
