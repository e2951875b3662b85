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
// once per call for every depth; each depth then needs two w-tap passes over the rows and columns
// its scale reaches, instead of four 2M-point FFTs per line.  The second pass is fused with the
// depth's transfer contraction Y_z(kappa) = sum_f Phat_{z,f}(kappa) Gs_z[class(kappa)][f].
#include <type_traits>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

__device__ __forceinline__ int wrap_mod(int m, int L) {
  const int r = m % L;
  return r < 0 ? r + L : r;
}

// P1[r][kx][f] = sum_t wt[kx][t] Yh[row(ylo + r)][col(m0[kx] + t)][f]: the x pass of one depth over
// the R rows its y taps reach.  Yh [L][L][F] at index m + L/2 (periodic in m); one thread per
// (r, kx) and FV adjacent channels (two as one 16-byte access when F is even), f fastest.
template <int FV>
__global__ void srsd_interp_x_kernel(const float2* __restrict__ Yh, int L, int M, int F, int ylo, int R, int w,
                                     const int* __restrict__ m0, const float* __restrict__ wt,
                                     float2* __restrict__ P1) {
  using V = typename std::conditional<FV == 2, float4, float2>::type;
  const int FG = F / FV;  // channel groups per (r, kx)
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)R * M * FG) return;
  const int fg = (int)(idx % FG);
  const long long rest = idx / FG;
  const int kx = (int)(rest % M), r = (int)(rest / M);
  const V* row = reinterpret_cast<const V*>(Yh + (size_t)wrap_mod(ylo + r + L / 2, L) * L * F) + fg;
  const int mb = __ldg(m0 + kx) + L / 2;
  const float* wk = wt + (size_t)kx * w;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  for (int t = 0; t < w; ++t) {
    const float c = __ldg(wk + t);
    const V v = __ldg(row + (size_t)wrap_mod(mb + t, L) * FG);
    a0 = fmaf(c, v.x, a0);
    a1 = fmaf(c, v.y, a1);
    if constexpr (FV == 2) {
      a2 = fmaf(c, v.z, a2);
      a3 = fmaf(c, v.w, a3);
    }
  }
  if constexpr (FV == 2)
    reinterpret_cast<float4*>(P1)[idx] = make_float4(a0, a1, a2, a3);
  else
    P1[idx] = make_float2(a0, a1);
}

// Y[k][z] = sum_f Gs_z[class(k)][f] * sum_t wt[ky][t] P1[m0[ky] + t - ylo][kx][f], k = (ky, kx):
// the y pass fused with the depth's contraction.  One warp per column kx and run of kYRun
// consecutive ky (consecutive warps take consecutive kx), lanes over f (F <= 32 * 8): ky and ky + 1
// share all but about 2 / s of their w rows, so a warp finds most of its P1 rows in L1.  The f sum
// is reduced by shuffles.
constexpr int kMaxFPerLane = 8;
constexpr int kYRun = 32;
template <int FPL>  // F <= 32 FPL
__global__ void srsd_interp_y_contract_kernel(const float2* __restrict__ P1, int M, int F, int Z, int z, int ylo,
                                              int w, const int* __restrict__ m0, const float* __restrict__ wt,
                                              const float2* __restrict__ Gs_z, float2* __restrict__ Y) {
  const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  const int nrun = (M + kYRun - 1) / kYRun;
  if (warp >= M * nrun) return;
  const int kxi = warp % M, run = warp / M;
  const int ax = abs(kxi - M / 2);
  const int ky1 = min(M, (run + 1) * kYRun);
  for (int kyi = run * kYRun; kyi < ky1; ++kyi) {
    const int ay = abs(kyi - M / 2), p = max(ax, ay), q = min(ax, ay);
    const float2* g = Gs_z + (size_t)(p * (p + 1) / 2 + q) * F;
    const int r0 = __ldg(m0 + kyi) - ylo;
    const float* wk = wt + (size_t)kyi * w;
    float2 ph[FPL];
#pragma unroll
    for (int j = 0; j < FPL; ++j) ph[j] = make_float2(0.f, 0.f);
    for (int t = 0; t < w; ++t) {
      const float c = __ldg(wk + t);
      const float2* row = P1 + ((size_t)(r0 + t) * M + kxi) * F;
#pragma unroll
      for (int j = 0; j < FPL; ++j) {
        const int f = lane + 32 * j;
        if (f < F) {
          const float2 v = __ldg(row + f);
          ph[j].x = fmaf(c, v.x, ph[j].x);
          ph[j].y = fmaf(c, v.y, ph[j].y);
        }
      }
    }
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < FPL; ++j) {
      const int f = lane + 32 * j;
      if (f < F) {
        const float2 gv = __ldg(g + f);
        acc.x = fmaf(ph[j].x, gv.x, fmaf(-ph[j].y, gv.y, acc.x));
        acc.y = fmaf(ph[j].x, gv.y, fmaf(ph[j].y, gv.x, acc.y));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) Y[((size_t)kyi * M + kxi) * Z + z] = acc;
  }
}

}  // namespace

cudaError_t launch_srsd_interp_x(const float2* Yh, int L, int M, int F, int ylo, int R, int w, const int* m0,
                                 const float* wt, float2* P1, cudaStream_t s) {
  const long long n = (long long)R * M * F;
  if (L < 2 || M < 2 || F < 1 || R < 1 || w < 1 || n >= (1LL << 40)) return cudaErrorInvalidValue;
  const int threads = 256;
  const bool pairs = F % 2 == 0;  // 16-byte accesses: Yh and P1 rows start on 16 bytes
  const long long blocks = (n / (pairs ? 2 : 1) + threads - 1) / threads;
  if (blocks >= (1LL << 31)) return cudaErrorInvalidValue;
  if (pairs)
    srsd_interp_x_kernel<2><<<(unsigned)blocks, threads, 0, s>>>(Yh, L, M, F, ylo, R, w, m0, wt, P1);
  else
    srsd_interp_x_kernel<1><<<(unsigned)blocks, threads, 0, s>>>(Yh, L, M, F, ylo, R, w, m0, wt, P1);
  return cudaGetLastError();
}

cudaError_t launch_srsd_interp_y_contract(const float2* P1, int M, int F, int Z, int z, int ylo, int w, const int* m0,
                                          const float* wt, const float2* Gs_z, float2* Y, cudaStream_t s) {
  if (M < 2 || F < 1 || F > 32 * kMaxFPerLane || z < 0 || z >= Z || w < 1) return cudaErrorInvalidValue;
  const long long threads_total = (long long)M * ((M + kYRun - 1) / kYRun) * 32;
  const int threads = 256;
  const unsigned blocks = (unsigned)((threads_total + threads - 1) / threads);
  if (F <= 32)
    srsd_interp_y_contract_kernel<1><<<blocks, threads, 0, s>>>(P1, M, F, Z, z, ylo, w, m0, wt, Gs_z, Y);
  else if (F <= 64)
    srsd_interp_y_contract_kernel<2><<<blocks, threads, 0, s>>>(P1, M, F, Z, z, ylo, w, m0, wt, Gs_z, Y);
  else if (F <= 128)
    srsd_interp_y_contract_kernel<4><<<blocks, threads, 0, s>>>(P1, M, F, Z, z, ylo, w, m0, wt, Gs_z, Y);
  else
    srsd_interp_y_contract_kernel<8><<<blocks, threads, 0, s>>>(P1, M, F, Z, z, ylo, w, m0, wt, Gs_z, Y);
  return cudaGetLastError();
}

}  // namespace nursd
