// Panel FFT: batched 1-D complex DFTs along a strided axis, CP channels per CTA.
//
// Every 2-D transform of the operator (the NUFFT fine-grid FFT of Sec. 6, the
// IFFT of Eq. 4, the transfer-function FFT{G}) is two of these passes over
// channel-last data, so each pass streams whole rows of CP contiguous complex
// values from HBM.  Inside the CTA the transform is a self-sorting Stockham
// radix-4 (plus one radix-2 pass for odd log2 n) in shared memory: each pass
// stages its butterflies in registers, synchronises, and writes the permuted
// results back, so one buffer of n*CP complex values suffices.
//
// Pruning: the input is a window of `nin` elements (the rest is zero) and only
// `nout` output bins are written, which is how the NUFFT keeps the central
// M modes of its 2M grid and the IFFT keeps the N x N crop.
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

template <bool INV>
__device__ __forceinline__ void bfly4(float2& v0, float2& v1, float2& v2, float2& v3) {
  const float2 a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = csub(v1, v3);
  // forward: X1 = b - i d, X3 = b + i d; inverse swaps the sign of i.
  const float2 m = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
  v0 = cadd(a, c);
  v2 = csub(a, c);
  v1 = cadd(b, m);
  v3 = csub(b, m);
}

template <bool INV>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int q) {
  float2 w = __ldg(tw + q);
  if (INV) w.y = -w.y;
  return w;
}

// One Stockham pass of radix R (2 or 4) at stride Ns (a power of two).
// Butterfly j (0 <= j < n/R) reads x[j + t n/R], applies e^{-+2 pi i (j mod Ns) t / (Ns R)},
// and writes x'[(j - j mod Ns) R + j mod Ns + t Ns].
template <int LOGN, int CP, int NT, int R, bool INV>
__device__ __forceinline__ void stockham_pass(float2* sm, int Ns, const float2* __restrict__ tw) {
  constexpr int n = 1 << LOGN;
  constexpr int SR = CP + 1;  // padded row stride: conflict-free for both load orders
  constexpr int NB = (n / R) * CP;
  constexpr int PER = (NB + NT - 1) / NT;
  float2 v[PER][R];
  const int twstride_log = kTwiddleLog - (__ffs(Ns * R) - 1);  // 2^12 / (Ns R)
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int jb = threadIdx.x + r * NT;
    if ((NB % NT == 0) || jb < NB) {
      const int j = jb / CP, q = jb % CP;
      const int k = j & (Ns - 1);
#pragma unroll
      for (int t = 0; t < R; ++t) v[r][t] = sm[(j + t * (n / R)) * SR + q];
      if (Ns > 1) {
#pragma unroll
        for (int t = 1; t < R; ++t) v[r][t] = cmul(v[r][t], twiddle<INV>(tw, (k * t) << twstride_log));
      }
      if (R == 4) {
        bfly4<INV>(v[r][0], v[r][1], v[r][2], v[r][3]);
      } else {
        const float2 a = v[r][0];
        v[r][0] = cadd(a, v[r][1]);
        v[r][1] = csub(a, v[r][1]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int jb = threadIdx.x + r * NT;
    if ((NB % NT == 0) || jb < NB) {
      const int j = jb / CP, q = jb % CP;
      const int k = j & (Ns - 1);
      const int o = (j - k) * R + k;
#pragma unroll
      for (int t = 0; t < R; ++t) sm[(o + t * Ns) * SR + q] = v[r][t];
    }
  }
  __syncthreads();
}

template <int LOGN, int CP, int NT, bool INV>
__global__ void __launch_bounds__(NT) panel_fft_kernel(const PanelArgs a) {
  constexpr int n = 1 << LOGN;
  constexpr int SR = CP + 1;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const int hi0 = (blockIdx.x / nlo) * a.CHI;
  const int lo0 = (blockIdx.x % nlo) * a.CLO;
  const int b = blockIdx.y;

  // ---- load the input window (zero elsewhere)
  const float2* __restrict__ inb = a.in + (long long)b * a.in_sb;
  for (int idx = tid; idx < a.nin * CP; idx += NT) {
    int i, q;
    if (a.load_i_fastest) {
      i = idx % a.nin;
      q = idx / a.nin;
    } else {
      i = idx / CP;
      q = idx % CP;
    }
    const int qh = q / a.CLO, ql = q % a.CLO;
    const int hi = hi0 + qh, lo = lo0 + ql;
    float2 v = make_float2(0.f, 0.f);
    if (hi < a.hi_total && lo < a.lo_total) {
      v = __ldg(inb + i * a.in_si + hi * a.in_shi + lo * a.in_slo);
      if (a.mul_i) {
        const float m = __ldg(a.mul_i + i);
        v.x *= m;
        v.y *= m;
      }
    }
    sm[((i + a.in_off) & (n - 1)) * SR + q] = v;
  }
  for (int idx = tid; idx < (n - a.nin) * CP; idx += NT) {
    const int j = idx / CP + a.nin, q = idx % CP;
    sm[((j + a.in_off) & (n - 1)) * SR + q] = make_float2(0.f, 0.f);
  }
  __syncthreads();

  // ---- transform
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < LOGN / 2; ++p) {
    stockham_pass<LOGN, CP, NT, 4, INV>(sm, Ns, a.twiddle);
    Ns <<= 2;
  }
  if (LOGN & 1) stockham_pass<LOGN, CP, NT, 2, INV>(sm, Ns, a.twiddle);

  // ---- store the selected bins
  const float sb = a.scale * (a.mul_b ? a.mul_b[b] : 1.f);
  for (int idx = tid; idx < a.nout * CP; idx += NT) {
    int o, qh, ql;
    if (a.store_o_fastest) {
      o = idx % a.nout;
      const int q = idx / a.nout;
      qh = q / a.CLO;
      ql = q % a.CLO;
    } else if (a.store_hi_fastest) {
      qh = idx % a.CHI;
      const int rest = idx / a.CHI;
      ql = rest % a.CLO;
      o = rest / a.CLO;
    } else {
      const int q = idx % CP;
      o = idx / CP;
      qh = q / a.CLO;
      ql = q % a.CLO;
    }
    const int hi = hi0 + qh, lo = lo0 + ql;
    if (hi >= a.hi_total || lo >= a.lo_total) continue;
    float2 v = sm[((o + a.out_off) & (n - 1)) * SR + qh * a.CLO + ql];
    const float s = sb * (a.mul_o ? __ldg(a.mul_o + o) : 1.f);
    v.x *= s;
    v.y *= s;
    const long long off = (long long)b * a.out_sb + (long long)o * a.out_si + (long long)hi * a.out_shi +
                          (long long)lo * a.out_slo;
    if (a.out_mag)
      a.out_mag[off] = sqrtf(v.x * v.x + v.y * v.y);
    else
      a.out[off] = v;
  }
}

// Scaled DFT by Bluestein's chirp-z (Supp. A.1): X[kappa] = c(kappa) sum_n (x[n] c(n)) b(kappa - n)
// with c(n) = e^{-pi i n^2 / (M s)}, b(d) = e^{+pi i d^2 / (M s)}.  The linear convolution is a
// circular one of length n = 2M >= 2M - 1: chirp the window, FFT, multiply by bhat = FFT(b)/n,
// inverse FFT, chirp the kept outputs.  cpre/cpost are per input / output index.
template <int LOGN, int CP, int NT>
__global__ void __launch_bounds__(NT, 2) panel_bluestein_kernel(const PanelArgs a, const float2* __restrict__ cpre,
                                                            const float2* __restrict__ bhat,
                                                            const float2* __restrict__ cpost) {
  constexpr int n = 1 << LOGN;
  constexpr int SR = CP + 1;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const int hi0 = (blockIdx.x / nlo) * a.CHI;
  const int lo0 = (blockIdx.x % nlo) * a.CLO;
  const int b = blockIdx.y;
  const float2* __restrict__ inb = a.in + (long long)b * a.in_sb;
  for (int idx = tid; idx < a.nin * CP; idx += NT) {
    const int i = idx / CP, q = idx % CP;
    const int qh = q / a.CLO, ql = q % a.CLO;
    const int hi = hi0 + qh, lo = lo0 + ql;
    float2 v = make_float2(0.f, 0.f);
    if (hi < a.hi_total && lo < a.lo_total) v = cmul(__ldg(inb + i * a.in_si + hi * a.in_shi + lo * a.in_slo), __ldg(cpre + i));
    sm[((i + a.in_off) & (n - 1)) * SR + q] = v;
  }
  for (int idx = tid; idx < (n - a.nin) * CP; idx += NT) {
    const int j = idx / CP + a.nin, q = idx % CP;
    sm[((j + a.in_off) & (n - 1)) * SR + q] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  int Ns = 1;
#pragma unroll
  for (int p = 0; p < LOGN / 2; ++p) {
    stockham_pass<LOGN, CP, NT, 4, false>(sm, Ns, a.twiddle);
    Ns <<= 2;
  }
  if (LOGN & 1) stockham_pass<LOGN, CP, NT, 2, false>(sm, Ns, a.twiddle);
  for (int idx = tid; idx < n * CP; idx += NT) {
    const int j = idx / CP, q = idx % CP;
    sm[j * SR + q] = cmul(sm[j * SR + q], __ldg(bhat + j));
  }
  __syncthreads();
  Ns = 1;
#pragma unroll
  for (int p = 0; p < LOGN / 2; ++p) {
    stockham_pass<LOGN, CP, NT, 4, true>(sm, Ns, a.twiddle);
    Ns <<= 2;
  }
  if (LOGN & 1) stockham_pass<LOGN, CP, NT, 2, true>(sm, Ns, a.twiddle);
  for (int idx = tid; idx < a.nout * CP; idx += NT) {
    const int q = idx % CP, o = idx / CP;
    const int qh = q / a.CLO, ql = q % a.CLO;
    const int hi = hi0 + qh, lo = lo0 + ql;
    if (hi >= a.hi_total || lo >= a.lo_total) continue;
    const float2 v = cmul(sm[((o + a.out_off) & (n - 1)) * SR + q], __ldg(cpost + o));
    a.out[(long long)b * a.out_sb + (long long)o * a.out_si + (long long)hi * a.out_shi + (long long)lo * a.out_slo] =
        v;
  }
}

template <int LOGN, int CP, int NT>
cudaError_t launch_bluestein_one(const PanelArgs& a, const float2* cpre, const float2* bhat, const float2* cpost,
                                 cudaStream_t s) {
  const size_t smem = sizeof(float2) * (size_t(1) << LOGN) * (CP + 1);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(panel_bluestein_kernel<LOGN, CP, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int nhi = (a.hi_total + a.CHI - 1) / a.CHI;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  dim3 grid(nhi * nlo, a.batch);
  panel_bluestein_kernel<LOGN, CP, NT><<<grid, NT, smem, s>>>(a, cpre, bhat, cpost);
  return cudaGetLastError();
}

template <int LOGN, int CP, int NT, bool INV>
cudaError_t launch_one(const PanelArgs& a, cudaStream_t s) {
  const size_t smem = sizeof(float2) * (size_t(1) << LOGN) * (CP + 1);
  static bool configured = false;  // one attribute call per instantiation and process
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(panel_fft_kernel<LOGN, CP, NT, INV>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int nhi = (a.hi_total + a.CHI - 1) / a.CHI;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  dim3 grid(nhi * nlo, a.batch);
  panel_fft_kernel<LOGN, CP, NT, INV><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, int CP, int NT>
cudaError_t launch_dir(bool inverse, const PanelArgs& a, cudaStream_t s) {
  return inverse ? launch_one<LOGN, CP, NT, true>(a, s) : launch_one<LOGN, CP, NT, false>(a, s);
}

}  // namespace

// Channels per CTA: 16 up to n = 512, then fewer so that a CTA's buffer stays
// near 68 KB and three CTAs share an SM (overlapping one's loads with another's
// transform).
// Lengths 512-2048 use the register-resident kernels of fft_reg.cu (512 threads,
// 16 / 8 / 4 channels); shorter ones this shared-memory Stockham kernel.
int panel_width(int logn) { return logn >= 9 ? panel_width_reg(logn) : 16; }

cudaError_t launch_panel_bluestein(int logn, const PanelArgs& a, const float2* cpre, const float2* bhat,
                                   const float2* cpost, cudaStream_t s) {
  if (a.CHI * a.CLO != panel_width(logn) || a.nin > (1 << logn) || a.nout > (1 << logn) || a.batch < 1 ||
      a.batch > 65535)
    return cudaErrorInvalidValue;
  if (logn >= 9) return launch_panel_bluestein_reg(logn, a, cpre, bhat, cpost, s);
  switch (logn) {
    case 5: return launch_bluestein_one<5, 16, 128>(a, cpre, bhat, cpost, s);
    case 6: return launch_bluestein_one<6, 16, 256>(a, cpre, bhat, cpost, s);
    case 7: return launch_bluestein_one<7, 16, 256>(a, cpre, bhat, cpost, s);
    case 8: return launch_bluestein_one<8, 16, 256>(a, cpre, bhat, cpost, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_panel_fft(int logn, bool inverse, const PanelArgs& a, cudaStream_t s) {
  if (a.CHI * a.CLO != panel_width(logn) || a.nin > (1 << logn) || a.nout > (1 << logn) || a.batch < 1)
    return cudaErrorInvalidValue;
  if (a.batch > 65535) {  // the batch is a grid dimension: launch it in chunks
    if (a.prod_g) return cudaErrorInvalidValue;  // its mode classes follow the batch index
    constexpr int kChunk = 32768;
    for (int b0 = 0; b0 < a.batch; b0 += kChunk) {
      PanelArgs c = a;
      c.batch = std::min(kChunk, a.batch - b0);
      c.in = a.in + b0 * a.in_sb;
      if (a.out) c.out = a.out + b0 * a.out_sb;
      if (a.out_mag) c.out_mag = a.out_mag + b0 * a.out_sb;
      if (a.mul_b) c.mul_b = a.mul_b + b0;
      const cudaError_t e = launch_panel_fft(logn, inverse, c, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  switch (logn) {
    case 3: return launch_dir<3, 16, 128>(inverse, a, s);
    case 4: return launch_dir<4, 16, 128>(inverse, a, s);
    case 5: return launch_dir<5, 16, 128>(inverse, a, s);
    case 6: return launch_dir<6, 16, 256>(inverse, a, s);
    case 7: return launch_dir<7, 16, 256>(inverse, a, s);
    case 8: {
      const cudaError_t e = launch_panel_fft32_256(inverse, a, s);
      if (e != cudaErrorNotSupported) return e;
      return launch_dir<8, 16, 256>(inverse, a, s);
    }
    case 9:
    case 10:
    case 11: return launch_panel_fft_reg(logn, inverse, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nursd
