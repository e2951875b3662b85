// Scaled DFT of SRSD (Sec. 4, Eq. SFFT) as a type-2 evaluation of one shared oversampled FFT.
//
// Along one axis the scaled DFT of x[n], n in I_M, is the DTFT at the frequencies 2 pi kappa / (M s),
//   X(kappa) = sum_n x[n] exp(-2 pi i kappa n / (M s)),  kappa in I_M,
// i.e. at coordinate u = L kappa / (M s) = 2 kappa / s of the L = 2M point grid.  With
// xh[m] = FFT_L[x / psi_hat][m] (psi_hat the Fourier transform of the ES kernel phi, the same
// deconvolution as the spatial NUFFT) the ES interpolation
//   X(kappa) ~ sum_{t < w} phi(2 (m0 + t - u) / w) xh[m0 + t],  m0 = ceil(u - w / 2),
// reproduces it to the kernel's accuracy (Poisson summation: exp(-2 pi i m n / L) summed against
// phi over m gives psi_hat(n) exp(-2 pi i u n / L)).  The 2D FFT of u / (psi_hat x psi_hat) is taken
// once per call for every depth; each depth then needs w x w taps over the block its scale
// reaches, instead of four 2M-point FFTs per line, taken in one pass together with the depth's
// transfer contraction Y_z(kappa) = sum_f Phat_{z,f}(kappa) Gs_z[class(kappa)][f].
#include "mbarrier.cuh"
#include "nursd_internal.cuh"

namespace nursd {
namespace {

__device__ __forceinline__ int wrap_mod(int m, int L) {
  const int r = m % L;
  return r < 0 ? r + L : r;
}

constexpr int kMaxFPerLane = 8;
constexpr int kYRun = 16;

// d = a * (b.x, b.y) + c as one packed fma.rn.f32x2 (the same scalar on both halves).
__device__ __forceinline__ float2 fma2s(float a, float2 b, float2 c) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %2};\n mov.b64 rb, {%3, %4};\n mov.b64 rc, {%5, %6};\n"
      " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
// The three steps of one depth in one pass, without the x-tapped rows in memory (every listed depth
// in one launch, blockIdx.y selecting it):
// Y[k][z] = sum_f Gs_z[class(k)][f] sum_ty wt[ky][ty] X[m0[ky] + ty][kx][f] with
// X[m][kx][f] = sum_tx wt[kx][tx] Yh[m][m0[kx] + tx][f].  One warp per column kx and run of kYRun
// consecutive ky, lanes over f (F <= 32 FPL).  The warp keeps X of the W rows its current ky needs
// in registers; the next ky starts at most two rows further (the tap tables must advance by at
// most two cells per mode: the coordinate 2 ky / s of SRSD advances by 2 / s <= 2 for scales >= 1),
// so at most two new rows are x-tapped per step.  Tap and contraction MACs are packed
// fma.rn.f32x2 on (re, im) pairs.
// FS = 2: the channels of a mode are split over two warps (channel block fs), each adding its part
// of the f sum to Y with an atomic add; Y starts at zero, and a sum of two terms onto zero does not
// depend on their order, so the result is reproducible.
template <int FPL, int W, int FS>
__global__ void srsd_interp_xy_contract_kernel(const float2* __restrict__ Yh, int L, int M, int F, int Z,
                                               const int* __restrict__ zlist, const int* __restrict__ m0_all,
                                               const float* __restrict__ wt_all, const float2* __restrict__ Gs,
                                               int ncls, float2* __restrict__ Y) {
  // blockIdx.y: the depth (an entry of zlist), its taps [M] / [M][W] and table [ncls][F]
  const int z = __ldg(zlist + blockIdx.y);
  const int* __restrict__ m0 = m0_all + (size_t)z * M;
  const float* __restrict__ wt = wt_all + (size_t)z * M * W;
  const float2* __restrict__ Gs_z = Gs + (size_t)z * ncls * F;
  const int gw = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  const int nrun = (M + kYRun - 1) / kYRun;
  if (gw >= M * nrun * FS) return;
  const int fs = gw % FS, warp = gw / FS;
  const int fbase = fs * 32 * FPL;  // this warp's channels: fbase + lane + 32 j, j < FPL
  const int kxi = warp % M, run = warp / M;
  const int ax = abs(kxi - M / 2);
  // x taps of this column: weights and the first column on the periodic 2M grid
  float cx[W];
#pragma unroll
  for (int t = 0; t < W; ++t) cx[t] = __ldg(wt + (size_t)kxi * W + t);
  const int cb = __ldg(m0 + kxi) + L / 2;
  auto xtap = [&](int m, float2 (&out)[FPL]) {  // X[m][kx][f] for the lane's channels
    const float2* row = Yh + (size_t)wrap_mod(m + L / 2, L) * L * F;
#pragma unroll
    for (int j = 0; j < FPL; ++j) out[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < W; ++t) {
      const float2* cell = row + (size_t)wrap_mod(cb + t, L) * F;
#pragma unroll
      for (int j = 0; j < FPL; ++j) {
        const int f = fbase + lane + 32 * j;
        if (f < F) out[j] = fma2s(cx[t], __ldg(cell + f), out[j]);
      }
    }
  };
  const int ky0 = run * kYRun, ky1 = min(M, ky0 + kYRun);
  float2 xr[W][FPL];  // X of rows rbase .. rbase + W - 1
  int rbase = __ldg(m0 + ky0);
#pragma unroll
  for (int r = 0; r < W; ++r) xtap(rbase + r, xr[r]);
  for (int kyi = ky0; kyi < ky1; ++kyi) {
    const int mk = __ldg(m0 + kyi);
    for (int d = mk - rbase; d > 0; --d) {  // slide the window by one row
#pragma unroll
      for (int r = 0; r + 1 < W; ++r)
#pragma unroll
        for (int j = 0; j < FPL; ++j) xr[r][j] = xr[r + 1][j];
      ++rbase;
      xtap(rbase + W - 1, xr[W - 1]);
    }
    const int ay = abs(kyi - M / 2), p = max(ax, ay), q = min(ax, ay);
    const float2* g = Gs_z + (size_t)(p * (p + 1) / 2 + q) * F;
    float cy[W];
#pragma unroll
    for (int t = 0; t < W; ++t) cy[t] = __ldg(wt + (size_t)kyi * W + t);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < FPL; ++j) {
      const int f = fbase + lane + 32 * j;
      float2 ph = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < W; ++t) ph = fma2s(cy[t], xr[t][j], ph);
      if (f < F) {  // acc += ph * g: (ph.x, ph.x) (gx, gy) + (ph.y, ph.y) (-gy, gx)
        const float2 gv = __ldg(g + f);
        acc = fma2s(ph.y, make_float2(-gv.y, gv.x), fma2s(ph.x, gv, acc));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
      float2* y = Y + ((size_t)kyi * M + kxi) * Z + z;
      if constexpr (FS == 1) {
        *y = acc;
      } else {
        atomicAdd(&y->x, acc.x);
        atomicAdd(&y->y, acc.y);
      }
    }
  }
}

// ------------------------------------------------------------------ staged-row form
// The same sums with the input rows staged in shared memory.  A CTA takes kTileX adjacent columns
// kx (one warp each, lanes over channel pairs 2 (lane + 32 j), j < NJ, so F <= 64 NJ) and a run of
// kRunY consecutive ky of one depth.  Its columns' taps cover nc <= 2 (kTileX - 1) + W consecutive
// cells of every row; a copy warp streams the rows the run's y taps reach (nr = m0[last ky] -
// m0[first ky] + W of them, in order) into a kRing-slot ring with cp.async.bulk: one contiguous
// copy of nc x F values per row (two where the span wraps around the periodic grid), completing on
// the slot's "full" barrier.  Every column warp x-taps each row once as it enters its window of W
// rows in registers and releases the slot on its "empty" barrier (one arrival per warp); so the
// cells a row's columns share are read from global memory once per CTA instead of once per column,
// and the loads run kRing rows ahead of the arithmetic.  Requires F even (16-byte copies).
// Every barrier wait is bounded: on time-out the CTA raises its abort flag and status bit 2, the
// other roles stop at their next wait, and the copy warp waits (bounded) for the copies it issued.
// A tap table that advances by more than two cells per mode (or backwards) would not fit the
// staged span: the CTA sets status bit 8 and writes nothing.
constexpr int kTileX = 8, kRunY = 64, kRing = 3;
constexpr int kTileThreads = (kTileX + 1) * 32;
constexpr long long kTileWait = 1LL << 22;

__host__ __device__ constexpr int tile_ncmax(int W) { return 2 * (kTileX - 1) + W; }
__host__ __device__ constexpr unsigned tile_head(int W) { return (64u + 4u * kRunY * (W + 1) + 127u) / 128u * 128u; }
// bytes of one ring slot: the widest span of F values plus the channels past F that lanes of the
// last pair block read (finite or not, they never reach Y)
__host__ __device__ inline unsigned tile_slot(int W, int F) {
  return ((unsigned)tile_ncmax(W) * F * 8u + 512u + 127u) / 128u * 128u;
}

// Wait for phase `parity` of `bar`: false once the CTA's abort flag is up, or after kTileWait polls
// (which raise it, with status bit 2).
__device__ __forceinline__ bool tile_wait(unsigned long long* bar, unsigned parity, volatile int* abort_flag,
                                          int* status) {
  for (long long it = 0; it < kTileWait; ++it) {
    if (mbar::test(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  atomicOr(status, 2);
  return false;
}

// two CTAs per SM (a 112-register cap measured 40 % slower than the 96 this bound gives)
template <int W, int NJ>
__global__ void __launch_bounds__(kTileThreads, 2)
    srsd_tile_kernel(const float2* __restrict__ Yh, int L, int M, int F, int Z, const int* __restrict__ zlist,
                     const int* __restrict__ m0_all, const float* __restrict__ wt_all,
                     const float2* __restrict__ Gs, int ncls, float2* __restrict__ Y, int* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned long long* full = reinterpret_cast<unsigned long long*>(sm);
  unsigned long long* empty = full + kRing;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + 48);
  int* info = reinterpret_cast<int*>(sm + 52);  // rows of the run, geometry ok
  int* m0y = reinterpret_cast<int*>(sm + 64);    // [kRunY] first y tap of each ky of the run
  float* cy = reinterpret_cast<float*>(m0y + kRunY);  // [kRunY][W] y weights
  unsigned char* ring = sm + tile_head(W);
  const unsigned slot_bytes = tile_slot(W, F);

  const int z = __ldg(zlist + blockIdx.y);
  const int* __restrict__ m0 = m0_all + (size_t)z * M;
  const float* __restrict__ wt = wt_all + (size_t)z * M * W;
  const float2* __restrict__ Gz = Gs + (size_t)z * ncls * F;
  const int ntx = (M + kTileX - 1) / kTileX;
  const int kx0 = (int)(blockIdx.x % ntx) * kTileX, ky0 = (int)(blockIdx.x / ntx) * kRunY;
  const int nkx = min(kTileX, M - kx0), nky = min(kRunY, M - ky0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  for (int i = threadIdx.x; i < nky; i += blockDim.x) m0y[i] = __ldg(m0 + ky0 + i);
  for (int i = threadIdx.x; i < nky * W; i += blockDim.x) cy[i] = __ldg(wt + (size_t)ky0 * W + i);
  if (threadIdx.x == 0) {
    for (int r = 0; r < kRing; ++r) {
      mbar::init(full + r, 1);
      mbar::init(empty + r, kTileX);
    }
    mbar::fence_init();
    *abort_flag = 0;
    bool ok = true;
    for (int i = 1; i < nkx; ++i) {
      const int d = __ldg(m0 + kx0 + i) - __ldg(m0 + kx0 + i - 1);
      ok = ok && d >= 0 && d <= 2;
    }
    for (int i = 1; i < nky; ++i) {
      const int d = __ldg(m0 + ky0 + i) - __ldg(m0 + ky0 + i - 1);
      ok = ok && d >= 0 && d <= 2;
    }
    const int nc = __ldg(m0 + kx0 + nkx - 1) - __ldg(m0 + kx0) + W;
    ok = ok && nc <= tile_ncmax(W) && nc <= L;
    info[0] = __ldg(m0 + ky0 + nky - 1) - __ldg(m0 + ky0) + W;
    info[1] = ok ? 1 : 0;
    if (!ok) atomicOr(status, 8);
  }
  __syncthreads();
  if (!info[1]) return;
  const int nr = info[0];
  const int cbase = __ldg(m0 + kx0);  // first staged cell (centred index)
  const int nc = __ldg(m0 + kx0 + nkx - 1) - cbase + W;

  if (warp == kTileX) {  // ---- copy warp (one thread)
    if (lane == 0) {
      const unsigned bytes = (unsigned)(nc * F * sizeof(float2));
      const int c = wrap_mod(cbase + L / 2, L);
      const int first = min(nc, L - c);  // cells before the span wraps
      int issued = 0;
      for (int r = 0; r < nr; ++r) {
        const int slot = r % kRing;
        if (r >= kRing && !tile_wait(empty + slot, ((r / kRing) - 1) & 1, abort_flag, status)) break;
        const float2* row = Yh + (size_t)wrap_mod(m0y[0] + r + L / 2, L) * L * F;
        unsigned char* dst = ring + (size_t)slot * slot_bytes;
        mbar::arrive_expect_tx(full + slot, bytes);
        mbar::copy_g2s(dst, row + (size_t)c * F, (unsigned)(first * F * sizeof(float2)), full + slot);
        if (first < nc)
          mbar::copy_g2s(dst + (size_t)first * F * sizeof(float2), row, (unsigned)((nc - first) * F * sizeof(float2)),
                         full + slot);
        issued = r + 1;
      }
      // the copies of the last issued rows must land before the CTA's shared memory is released
      for (int r = max(0, issued - kRing); r < issued; ++r) {
        long long it = 0;
        while (!mbar::test(full + r % kRing, (r / kRing) & 1) && ++it < kTileWait) {
        }
      }
    }
    return;
  }

  // ---- column warp
  const int kxi = kx0 + min(warp, nkx - 1);  // warps past the last column track it and store nothing
  const bool store = warp < nkx;
  float cx[W];
#pragma unroll
  for (int t = 0; t < W; ++t) cx[t] = __ldg(wt + (size_t)kxi * W + t);
  const int off = __ldg(m0 + kxi) - cbase;  // this column's first cell within the staged span
  const int ax = abs(kxi - M / 2);
  int taken = 0;
  // X of the next row for the lane's channel pairs; false when the CTA gives up
  auto take = [&](float4 (&out)[NJ]) -> bool {
    const int slot = taken % kRing;
    const bool ok = __all_sync(0xffffffffu, tile_wait(full + slot, (taken / kRing) & 1, abort_flag, status));
    if (!ok) return false;
    const float2* base = reinterpret_cast<const float2*>(ring + (size_t)slot * slot_bytes) + (size_t)off * F;
#pragma unroll
    for (int j = 0; j < NJ; ++j) out[j] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int t = 0; t < W; ++t) {
      const float4* cell = reinterpret_cast<const float4*>(base + (size_t)t * F);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const float4 v = cell[lane + 32 * j];
        const float2 lo = fma2s(cx[t], make_float2(v.x, v.y), make_float2(out[j].x, out[j].y));
        const float2 hi = fma2s(cx[t], make_float2(v.z, v.w), make_float2(out[j].z, out[j].w));
        out[j] = make_float4(lo.x, lo.y, hi.x, hi.y);
      }
    }
    __syncwarp();
    if (lane == 0) mbar::arrive(empty + slot);
    ++taken;
    return true;
  };
  float4 xr[W][NJ];  // X of rows rb .. rb + W - 1 (relative to the run's first row)
#pragma unroll
  for (int r = 0; r < W; ++r)
    if (!take(xr[r])) return;
  int rb = 0;
  // four consecutive ky at a time: their sums over f are reduced together (a reduce-scatter over
  // the lanes, three shuffles per mode instead of ten, and four independent chains)
  const int o = (lane >> 3) & 3;  // the ky of the group whose sum this lane ends with
  for (int kb = 0; kb < nky; kb += 4) {
    float2 acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      acc[i] = make_float2(0.f, 0.f);
      const int kyl = kb + i;
      if (kyl >= nky) continue;  // warp-uniform
      const int kyi = ky0 + kyl;
      const int ay = abs(kyi - M / 2), p = max(ax, ay), q = min(ax, ay);
      const float4* g = reinterpret_cast<const float4*>(Gz + (size_t)(p * (p + 1) / 2 + q) * F);
      float4 gv[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int ch = 2 * (lane + 32 * j);
        gv[j] = ch < F ? __ldg(g + lane + 32 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int need = m0y[kyl] - m0y[0]; rb < need; ++rb) {  // slide the window by one row
#pragma unroll
        for (int r = 0; r + 1 < W; ++r)
#pragma unroll
          for (int j = 0; j < NJ; ++j) xr[r][j] = xr[r + 1][j];
        if (!take(xr[W - 1])) return;
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (2 * (lane + 32 * j) < F) {
          float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
          for (int t = 0; t < W; ++t) {
            const float w_ = cy[kyl * W + t];
            lo = fma2s(w_, make_float2(xr[t][j].x, xr[t][j].y), lo);
            hi = fma2s(w_, make_float2(xr[t][j].z, xr[t][j].w), hi);
          }
          // acc += lo * g_lo + hi * g_hi (complex)
          acc[i] = fma2s(lo.x, make_float2(gv[j].x, gv[j].y), acc[i]);
          acc[i] = fma2s(lo.y, make_float2(-gv[j].y, gv[j].x), acc[i]);
          acc[i] = fma2s(hi.x, make_float2(gv[j].z, gv[j].w), acc[i]);
          acc[i] = fma2s(hi.y, make_float2(-gv[j].w, gv[j].z), acc[i]);
        }
      }
    }
    // reduce-scatter: lanes with bit 4 set keep ky 2, 3 (else 0, 1), then bit 3 picks one of the
    // two; after the last three butterflies lane 8 o holds the whole sum of ky kb + o
    const bool b4 = lane & 16, b3 = lane & 8;
    float2 w2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float2 send = b4 ? acc[i] : acc[i + 2], keep = b4 ? acc[i + 2] : acc[i];
      w2[i] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 16),
                          keep.y + __shfl_xor_sync(0xffffffffu, send.y, 16));
    }
    const float2 send = b3 ? w2[0] : w2[1], keep = b3 ? w2[1] : w2[0];
    float2 v = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, 8),
                           keep.y + __shfl_xor_sync(0xffffffffu, send.y, 8));
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    if ((lane & 7) == 0 && store && kb + o < nky) Y[((size_t)(ky0 + kb + o) * M + kxi) * Z + z] = v;
  }
}

template <int NJ>
cudaError_t tile_width(const float2* Yh, int L, int M, int F, int Z, const int* zlist, int nz, int w, const int* m0,
                       const float* wt, const float2* Gs, int ncls, float2* Y, int* status, cudaStream_t s) {
  const int ntx = (M + kTileX - 1) / kTileX, nrun = (M + kRunY - 1) / kRunY;
  const dim3 grid((unsigned)(ntx * nrun), (unsigned)nz);
  const size_t smem = tile_head(w) + (size_t)kRing * tile_slot(w, F);
  switch (w) {
#define NURSD_TILE(W_)                                                                                        \
  case W_: {                                                                                                  \
    static size_t configured = 0;                                                                             \
    if (smem > configured) {                                                                                  \
      const cudaError_t e =                                                                                   \
          cudaFuncSetAttribute(srsd_tile_kernel<W_, NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
      if (e != cudaSuccess) return e;                                                                         \
      configured = smem;                                                                                      \
    }                                                                                                         \
    srsd_tile_kernel<W_, NJ><<<grid, kTileThreads, smem, s>>>(Yh, L, M, F, Z, zlist, m0, wt, Gs, ncls, Y, status); \
    return cudaGetLastError();                                                                                \
  }
    NURSD_TILE(4) NURSD_TILE(5) NURSD_TILE(6) NURSD_TILE(7) NURSD_TILE(8)
#undef NURSD_TILE
    default:
      return cudaErrorInvalidValue;
  }
}

// The staged-row form serves even F <= 128 on grids at least two staged spans wide.
bool tile_form(int F, int L, int w) { return F % 2 == 0 && F <= 128 && L >= 2 * tile_ncmax(w); }

template <int FPL, int FS>
cudaError_t xy_width(const float2* Yh, int L, int M, int F, int Z, const int* zlist, int nz, int w, const int* m0,
                     const float* wt, const float2* Gs, int ncls, float2* Y, unsigned blocks, cudaStream_t s) {
  const dim3 grid(blocks, (unsigned)nz);
  switch (w) {
#define NURSD_XY(W_)                                                                                          \
  case W_:                                                                                                  \
    srsd_interp_xy_contract_kernel<FPL, W_, FS><<<grid, 64, 0, s>>>(Yh, L, M, F, Z, zlist, m0, wt, Gs, ncls, Y); \
    return cudaGetLastError();
    NURSD_XY(4) NURSD_XY(5) NURSD_XY(6) NURSD_XY(7) NURSD_XY(8)
#undef NURSD_XY
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace

bool srsd_interp_adds(int F, int L, int w) { return F > 64 && !tile_form(F, L, w); }

cudaError_t launch_srsd_interp_xy_contract(const float2* Yh, int L, int M, int F, int Z, const int* zlist, int nz,
                                           int w, const int* m0, const float* wt, const float2* Gs, int ncls,
                                           float2* Y, int* status, cudaStream_t s) {
  if (nz <= 0) return cudaSuccess;
  if (L < 2 || M < 2 || F < 1 || F > 32 * kMaxFPerLane || nz > 65535 || !zlist || w < 4 || w > 8 || !status)
    return cudaErrorInvalidValue;
  if (tile_form(F, L, w)) {
    if (F <= 64) return tile_width<1>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, status, s);
    return tile_width<2>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, status, s);
  }
  // above 64 channels a mode's channels are split over two warps (FS = 2: Y must be zero on entry)
  const int FS = F > 64 ? 2 : 1;
  const long long threads_total = (long long)M * ((M + kYRun - 1) / kYRun) * 32 * FS;
  // two warps per block: more resident warps at the registers of the register-held window
  const unsigned blocks = (unsigned)((threads_total + 63) / 64);
  if (F <= 32) return xy_width<1, 1>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, blocks, s);
  if (F <= 64) return xy_width<2, 1>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, blocks, s);
  if (F <= 128) return xy_width<2, 2>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, blocks, s);
  return xy_width<4, 2>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, blocks, s);
}

}  // namespace nursd
