// NUFFT type-1 spreading (Sec. 6, step 1): b[g][f] = sum_l P[l][f] phi_x phi_y.
//
// No atomics: one CTA owns a tile of the fine-grid window 16 cells wide and ROWS
// (4, 8 or 16, a plan setting) rows high, for 32 or 64 channels; each of its ROWS warps owns one tile
// row, each lane one channel (two adjacent ones when F is even and at least 64), and the row's 16
// cells live in registers.  Samples are binned by (tile column,
// edge flag, first footprint row), tile column major, the edge flag marking
// footprints that cross into the next tile column.  So the samples that touch
// the tile -- first rows ty*ROWS-w+1 .. ty*ROWS+ROWS-1 in this tile column, and in the
// edge part of the column to its left (a footprint of w <= 8 cells crosses at
// most one tile edge) -- are three contiguous slot ranges, none holding a sample
// that misses the tile.  The CTA stages them in shared memory in chunks (the 32
// channels of each sample's phasor, its footprint origin, its y weights and its
// x weights laid out on the tile's 16 cells, zero where the footprint misses a
// cell) -- one round of loads when P is already in sorted-slot order, two when
// its rows are found through the sorted index -- and the warp for row y adds the
// samples whose first row is in y-w+1 .. y (again contiguous sub-ranges) with
// packed two-lane FMAs over each 8-cell half of its row that the footprint
// reaches: no branch on where the footprint starts.  Every window cell is
// written exactly once, and the summation order is the sorted order, so results
// are reproducible run to run.
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int kCap = 128;      // samples staged per chunk
constexpr int kSeg = 8;        // cells per segment of a tile row that a visit skips when the footprint misses it

// Cells of the tile row in packed pairs: for cell 2j + h, lane-wise, acc_re[j] holds the real part
// in component h and acc_im[j] the imaginary part, so one fma.rn.f32x2 updates two cells.
constexpr int kPairs = kTile / 2;
constexpr int kRowPad = 8;                // x-weight row: cell c of the tile at index kRowPad + c
constexpr int kRowLen = kRowPad + kTile;  // 24 floats; indices below kRowPad are never read

template <int CPL>  // channels per lane; a CTA covers 32 CPL channels
struct SpreadSmem {
  float2 p[kCap][32 * CPL];  // phasor slices
  float wx[kCap][kRowLen];  // x weight of each tile cell (0 where the footprint misses it)
  float wy[kCap][8];      // y weights
  int2 org[kCap];         // segments of the tile row reached (bit h: cells kSeg h .. kSeg h + kSeg - 1), first row rel. to the tile's
  int l[kCap];            // sample index (row of P)
};

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 16 : 0) : "memory");
}
// The CPL channels of this lane's phasor slice of staged sample s: one copy of 8 CPL bytes.
template <int CPL>
__device__ __forceinline__ void copy_slice(float2* dst, const float2* src, bool valid) {
  if constexpr (CPL == 1)
    cp_async8(dst, src, valid);
  else
    cp_async16(dst, src, valid);
}

// d = a * b + c, lane-wise on two fp32 values, one instruction.
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
      " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}

// One CTA per (tile, group of 32 CPL channels); warp = tile row, lane = CPL adjacent channels.  A
// staged sample carries its x weights laid out on the tile's 16 cells (zeros outside its
// footprint), so the warp adds it to every cell of its row with 16 packed FMAs per channel and no
// branch on the offset; a zero weight leaves a cell's sum unchanged, so the result equals the
// footprint-only sum.  With CPL = 2 a visit's shared loads of the sample's weights serve twice
// the channels.
template <int KW, int kRows, bool BATCH, int CPL>
__global__ void __launch_bounds__(kRows * 32, (CPL == 1 ? 32 : 16) / kRows) spread_kernel(const float2* __restrict__ P, int F,
                                                                const int* __restrict__ bin_start,
                                                                const int* __restrict__ sorted_l,
                                                                const int2* __restrict__ i0,
                                                                const float* __restrict__ wts, int tiles, int W,
                                                                float2* __restrict__ fine, const SpreadItems it) {
  extern __shared__ __align__(16) unsigned char raw[];
  if constexpr (BATCH) {  // item blockIdx.z of a batched call: its phasors, sorted samples, bins and window
    const long long item = blockIdx.z;
    P += item * it.p_stride;
    bin_start += item * it.bstride;
    if (sorted_l) sorted_l += item * it.pts;
    i0 += item * it.pts;
    wts += item * it.pts * 2 * KW;
    fine += item * it.fine_stride;
  }
  SpreadSmem<CPL>& sm = *reinterpret_cast<SpreadSmem<CPL>*>(raw);
  constexpr int kCh = 32 * CPL;
  pdl_wait();  // the phasors, sorted samples and bins come from the kernels before
  pdl_trigger();
  constexpr int kWarps = kRows;  // one warp per tile row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ty = blockIdx.x / tiles, tx = blockIdx.x % tiles;
  const int f0 = blockIdx.y * kCh;
  const int y = ty * kRows + warp, col0 = tx * kTile;
  // Slot ranges over first rows rlo .. rhi (bin = (column * 2 + edge) * W + row): the left
  // column's edge part (every such footprint reaches this tile), then this column's interior
  // and edge parts; v indexes their concatenation.
  const int rlo = max(ty * kRows - KW + 1, 0), rhi1 = ty * kRows + kRows;
  const int* bsA = bin_start + ((tx - 1) * 2 + 1) * W;  // read only when tx > 0
  const int* bsB = bin_start + (tx * 2) * W;
  const int* bsC = bin_start + (tx * 2 + 1) * W;
  const int aS = tx > 0 ? bsA[rlo] : 0, nA = tx > 0 ? bsA[rhi1] - aS : 0;
  const int bS = bsB[rlo], nB = bsB[rhi1] - bS;
  const int cS = bsC[rlo], nAB = nA + nB;
  const int n = nAB + bsC[rhi1] - cS;
  // this warp's samples (first rows wlo .. y) in each range, as indices v
  const int wlo = max(y - KW + 1, 0);
  int2 wr[3];
  wr[0] = tx > 0 ? make_int2(bsA[wlo] - aS, bsA[y + 1] - aS) : make_int2(0, 0);
  wr[1] = make_int2(nA + bsB[wlo] - bS, nA + bsB[y + 1] - bS);
  wr[2] = make_int2(nAB + bsC[wlo] - cS, nAB + bsC[y + 1] - cS);
  auto slot_of = [&](int v) { return v < nA ? aS + v : (v < nAB ? bS + (v - nA) : cS + (v - nAB)); };
  // 3D slices: does the sample's z footprint reach this item's cell (the test the slice phasors use)?
  auto z_reaches = [&](int slot) {
    const float zz = 2.f * ((float)(it.gz_first + (int)blockIdx.z) - __ldg(it.uz + slot)) / (float)KW;
    return fabsf(zz) < 1.f;
  };

  float2 acc_re[kPairs][CPL], acc_im[kPairs][CPL];
#pragma unroll
  for (int j = 0; j < kPairs; ++j)
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      acc_re[j][c] = make_float2(0.f, 0.f);
      acc_im[j][c] = make_float2(0.f, 0.f);
    }
  const int fl = f0 + lane * CPL;  // this lane's first channel; CPL = 2 needs F even (whole pairs)
  const bool live = fl < F;
  for (int c0 = 0; c0 < n; c0 += kCap) {
    const int cn = min(kCap, n - c0);
    __syncthreads();  // the previous chunk has been consumed
    // one thread per sample (all loads in flight at once): index, origin, weights; when P is in
    // slot order its copies need no index and start here too
    if (!sorted_l)
      for (int s = warp; s < cn; s += kWarps) {
        const int slot = slot_of(c0 + s);
        const bool use = live && (!BATCH || !it.uz || z_reaches(slot));
        copy_slice<CPL>(&sm.p[s][lane * CPL], use ? P + (size_t)slot * F + fl : P, use);
      }
    for (int s = threadIdx.x; s < cn; s += kWarps * 32) {
      const int slot = slot_of(c0 + s);
      const int l = sorted_l ? __ldg(sorted_l + slot) : slot;
      const int2 o = __ldg(i0 + slot);
      const float* w = wts + (size_t)slot * 2 * KW;
      float wv[2 * KW];
#pragma unroll
      for (int t = 0; t < 2 * KW; ++t) wv[t] = __ldg(w + t);
      const int ox = o.x - col0;
      // segments of the tile row that the footprint ox .. ox+w-1 reaches (at least one)
      int halves = 0;
#pragma unroll
      for (int h = 0; h < kTile / kSeg; ++h) halves |= (ox < kSeg * (h + 1) && ox + KW > kSeg * h ? 1 : 0) << h;
      const int oy = o.y - ty * kRows;
      if (!NURSD_CHECK(oy > -KW && oy < kRows && ox > -KW && ox < kTile, it.status)) halves = 0;
      if (BATCH && it.uz && !z_reaches(slot)) halves = 0;  // a zero phasor in this slice: nothing to add
      sm.l[s] = l;
      sm.org[s] = make_int2(halves, oy);
      float4* row = reinterpret_cast<float4*>(&sm.wx[s][0]);
#pragma unroll
      for (int q = 0; q < kRowLen / 4; ++q) row[q] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int t = 0; t < KW; ++t) {
        const int c = kRowPad + ox + t;  // cells left of the tile fall below kRowPad, right of it past the row
        if (c >= 0 && c < kRowLen) sm.wx[s][c] = wv[t];
        sm.wy[s][t] = wv[KW + t];
      }
    }
    if (sorted_l) {  // the phasor rows are found through the sample indices just stored
      __syncthreads();
      for (int s = warp; s < cn; s += kWarps)
        copy_slice<CPL>(&sm.p[s][lane * CPL], live ? P + (size_t)sm.l[s] * F + fl : P, live);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int c1 = c0 + cn;
    auto visit = [&](int s, int2 og) {
      const float wyv = sm.wy[s][warp - og.y];  // the warp's row is footprint row warp - oy (0 .. w-1)
      float2 pv[CPL];
      if constexpr (CPL == 1) {
        pv[0] = sm.p[s][lane];
      } else {
        const float4 t = *reinterpret_cast<const float4*>(&sm.p[s][lane * 2]);
        pv[0] = make_float2(t.x, t.y);
        pv[1] = make_float2(t.z, t.w);
      }
      float2 re[CPL], im[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        re[c] = make_float2(pv[c].x * wyv, pv[c].x * wyv);
        im[c] = make_float2(pv[c].y * wyv, pv[c].y * wyv);
      }
      const float4* row = reinterpret_cast<const float4*>(&sm.wx[s][kRowPad]);
#pragma unroll
      for (int h = 0; h < kTile / kSeg; ++h) {
        if (og.x & (1 << h)) {  // warp-uniform: this segment of the row is reached
#pragma unroll
          for (int q = h * kSeg / 4; q < (h + 1) * kSeg / 4; ++q) {
            const float4 wq = row[q];
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
              acc_re[2 * q][c] = pfma(re[c], make_float2(wq.x, wq.y), acc_re[2 * q][c]);
              acc_im[2 * q][c] = pfma(im[c], make_float2(wq.x, wq.y), acc_im[2 * q][c]);
              acc_re[2 * q + 1][c] = pfma(re[c], make_float2(wq.z, wq.w), acc_re[2 * q + 1][c]);
              acc_im[2 * q + 1][c] = pfma(im[c], make_float2(wq.z, wq.w), acc_im[2 * q + 1][c]);
            }
          }
        }
      }
    };
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int s1 = min(wr[r].y, c1) - c0;
#pragma unroll 2  // two visits in flight: the next one's shared loads overlap this one's FMAs
      for (int s = max(wr[r].x, c0) - c0; s < s1; ++s) visit(s, sm.org[s]);
    }
  }
  if (live) {
    float2* dst = fine + ((size_t)y * W + col0) * F + fl;
#pragma unroll
    for (int j = 0; j < kPairs; ++j) {
      if constexpr (CPL == 1) {
        dst[(size_t)(2 * j) * F] = make_float2(acc_re[j][0].x, acc_im[j][0].x);
        dst[(size_t)(2 * j + 1) * F] = make_float2(acc_re[j][0].y, acc_im[j][0].y);
      } else {
        *reinterpret_cast<float4*>(dst + (size_t)(2 * j) * F) =
            make_float4(acc_re[j][0].x, acc_im[j][0].x, acc_re[j][1].x, acc_im[j][1].x);
        *reinterpret_cast<float4*>(dst + (size_t)(2 * j + 1) * F) =
            make_float4(acc_re[j][0].y, acc_im[j][0].y, acc_re[j][1].y, acc_im[j][1].y);
      }
    }
  }
}

template <int KW, int kRows, int CPL>
cudaError_t launch_cpl(const float2* P, int F, const int* bin_start, const int* sorted_l, const int2* i0,
                       const float* wts, int tiles, int W, float2* fine, const SpreadItems& it, cudaStream_t s) {
  const size_t smem = sizeof(SpreadSmem<CPL>);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(spread_kernel<KW, kRows, false, CPL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(spread_kernel<KW, kRows, true, CPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid((W / kRows) * tiles, (F + 32 * CPL - 1) / (32 * CPL), it.n);
  if (it.n > 1)
    return launch_pdl(spread_kernel<KW, kRows, true, CPL>, grid, dim3(kRows * 32), smem, s, P, F, bin_start, sorted_l,
                      i0, wts, tiles, W, fine, it);
  return launch_pdl(spread_kernel<KW, kRows, false, CPL>, grid, dim3(kRows * 32), smem, s, P, F, bin_start, sorted_l,
                    i0, wts, tiles, W, fine, it);
}

// Two channels per lane where the channels come in whole pairs and fill at least one 64-channel group
// (at 65,536 samples, F = 128: 0.130 vs 0.146 ms for one channel per lane).
template <int KW, int kRows>
cudaError_t launch_kw(const float2* P, int F, const int* bin_start, const int* sorted_l, const int2* i0,
                      const float* wts, int tiles, int W, float2* fine, const SpreadItems& it, cudaStream_t s) {
  if (F % 2 == 0 && F >= 64)
    return launch_cpl<KW, kRows, 2>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, it, s);
  return launch_cpl<KW, kRows, 1>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, it, s);
}

template <int KW>
cudaError_t launch_rows(const float2* P, int F, const int* bin_start, const int* sorted_l, const int2* i0,
                        const float* wts, int tiles, int W, float2* fine, int rows, const SpreadItems& it,
                        cudaStream_t s) {
  switch (rows) {
    case 4: return launch_kw<KW, 4>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, it, s);
    case 16: return launch_kw<KW, 16>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, it, s);
    default: return launch_kw<KW, 8>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, it, s);
  }
}

}  // namespace

bool spread_rows_supported(int rows) { return rows == 4 || rows == 8 || rows == 16; }

cudaError_t launch_spread(const float2* P, int F, const int* bin_start, const int* sorted_l, const int2* i0,
                          const float* wts, int width, int tiles, int W, float2* fine, cudaStream_t s, int rows,
                          const SpreadItems& it) {
  if (W != tiles * kTile || !spread_rows_supported(rows) || W % rows != 0 || it.n < 1 || it.n > 65535)
    return cudaErrorInvalidValue;
  switch (width) {
    case 4: return launch_rows<4>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, rows, it, s);
    case 5: return launch_rows<5>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, rows, it, s);
    case 6: return launch_rows<6>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, rows, it, s);
    case 7: return launch_rows<7>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, rows, it, s);
    case 8: return launch_rows<8>(P, F, bin_start, sorted_l, i0, wts, tiles, W, fine, rows, it, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nursd
