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

bool srsd_interp_adds(int F) { return F > 64; }

cudaError_t launch_srsd_interp_xy_contract(const float2* Yh, int L, int M, int F, int Z, const int* zlist, int nz,
                                           int w, const int* m0, const float* wt, const float2* Gs, int ncls,
                                           float2* Y, cudaStream_t s) {
  if (nz <= 0) return cudaSuccess;
  if (L < 2 || M < 2 || F < 1 || F > 32 * kMaxFPerLane || nz > 65535 || !zlist) return cudaErrorInvalidValue;
  // above 64 channels a mode's channels are split over two warps (FS = 2: Y must be zero on entry)
  const int FS = srsd_interp_adds(F) ? 2 : 1;
  const long long threads_total = (long long)M * ((M + kYRun - 1) / kYRun) * 32 * FS;
  // two warps per block: more resident warps at the registers of the register-held window
  const unsigned blocks = (unsigned)((threads_total + 63) / 64);
  if (F <= 32) return xy_width<1, 1>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, blocks, s);
  if (F <= 64) return xy_width<2, 1>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, blocks, s);
  if (F <= 128) return xy_width<2, 2>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, blocks, s);
  return xy_width<4, 2>(Yh, L, M, F, Z, zlist, nz, w, m0, wt, Gs, ncls, Y, blocks, s);
}

}  // namespace nursd
