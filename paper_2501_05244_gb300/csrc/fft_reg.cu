// Register-resident panel FFT for the long transforms (n = 512, 1024, 2048).
//
// Same contract as panel_fft_kernel (PanelArgs: a window of nin inputs placed
// at (i + in_off) mod n, nout bins kept at (o + out_off) mod n, CP channels per
// CTA), but each thread keeps 16 complex values in registers and the transform
// is three self-sorting Stockham stages of radix 16, 16 and n/256.  Inputs go
// straight from global memory into registers, outputs straight back, and the
// data crosses shared memory only between stages: two exchanges per transform
// instead of a shared-memory round trip per radix-4 pass.
//
// Stage s (radix R, stride Ns) maps butterfly j: inputs x[j + t n/R],
// twiddle e^{-+2 pi i (j mod Ns) t / (Ns R)}, outputs x'[(j - j mod Ns) R + j mod Ns + t Ns].
// With T = n/16 threads per transform, thread j0 does butterfly j0 of stages 1
// and 2 and butterflies j0 + m T (m < 16/R3) of stage 3, whose outputs are the
// final bins j + 256 t.
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr float kC8 = 0.70710678118654752440f;  // cos(pi/4)
constexpr float kC16 = 0.92387953251128675613f; // cos(pi/8)
constexpr float kS16 = 0.38268343236508977173f; // sin(pi/8)

template <bool INV>
__device__ __forceinline__ float2 mul_negi(float2 d) {  // forward: -i d; inverse: +i d
  return INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = mul_negi<INV>(csub(x1, x3));
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

// e^{-+2 pi i m / 16} for m = 1, 2, 3 (constants of the regular 16-gon)
template <bool INV>
__device__ __forceinline__ float2 w16(int m) {
  const float s = INV ? 1.f : -1.f;
  switch (m) {
    case 1: return make_float2(kC16, s * kS16);
    case 2: return make_float2(kC8, s * kC8);
    case 3: return make_float2(kS16, s * kC16);
    case 4: return make_float2(0.f, s);
    case 6: return make_float2(-kC8, s * kC8);
    case 9: return make_float2(-kC16, -s * kS16);
    default: return make_float2(1.f, 0.f);
  }
}

// In-place 16-point DFT: out[k1 + 4 k2] = sum_n x[n] W16^{n k}, via 4 x 4.
template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  float2 y[16];
#pragma unroll
  for (int s = 0; s < 4; ++s) {  // DFT over r of x[s + 4r] -> y[s][k1]
    float2 a = v[s], b = v[s + 4], c = v[s + 8], d = v[s + 12];
    dft4<INV>(a, b, c, d);
    y[s * 4 + 0] = a;
    y[s * 4 + 1] = b;
    y[s * 4 + 2] = c;
    y[s * 4 + 3] = d;
  }
#pragma unroll
  for (int s = 1; s < 4; ++s)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) y[s * 4 + k1] = cmul(y[s * 4 + k1], w16<INV>(s * k1));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {  // DFT over s -> X[k1 + 4 k2]
    float2 a = y[k1], b = y[4 + k1], c = y[8 + k1], d = y[12 + k1];
    dft4<INV>(a, b, c, d);
    v[k1] = a;
    v[k1 + 4] = b;
    v[k1 + 8] = c;
    v[k1 + 12] = d;
  }
}

// 8-point DFT of v[0..7] (out[k] in place), via 2 x 4.
template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const float s = INV ? 1.f : -1.f;
  o1 = cmul(o1, make_float2(kC8, s * kC8));
  o2 = cmul(o2, make_float2(0.f, s));
  o3 = cmul(o3, make_float2(-kC8, s * kC8));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

template <bool INV>
__device__ __forceinline__ float2 tw(const float2* __restrict__ table, int q) {
  float2 w = __ldg(table + (q & ((1 << kTwiddleLog) - 1)));
  if (INV) w.y = -w.y;
  return w;
}

// The transform on registers v[16] of thread j0 (channel column q of a panel with row stride SR).
// Entry: v[t] = x[j0 + t n/16].  Exit: v[m R3 + t] = X[j0 + m T + 256 t].
template <int LOGN, int SR, bool INV>
__device__ __forceinline__ void fft_core(float2* v, float2* sm, int j0, int q, const float2* __restrict__ table) {
  constexpr int n = 1 << LOGN;
  constexpr int T = n / 16;
  constexpr int R3 = n / 256;
  // stage 1: radix 16, Ns = 1
  dft16<INV>(v);
#pragma unroll
  for (int t = 0; t < 16; ++t) sm[(16 * j0 + t) * SR + q] = v[t];
  __syncthreads();
  // stage 2: radix 16, Ns = 16, twiddle e^{-+2 pi i (j0 mod 16) t / 256}
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = sm[(j0 + t * T) * SR + q];
  {
    const int k = j0 & 15;
#pragma unroll
    for (int t = 1; t < 16; ++t) v[t] = cmul(v[t], tw<INV>(table, (k * t) << (kTwiddleLog - 8)));
  }
  dft16<INV>(v);
  __syncthreads();
  {
    const int k = j0 & 15;
    const int base = (j0 - k) * 16 + k;
#pragma unroll
    for (int t = 0; t < 16; ++t) sm[(base + 16 * t) * SR + q] = v[t];
  }
  __syncthreads();
  // stage 3: radix R3, Ns = 256, butterflies j = j0 + m T (j < 256): inputs x[j + t 256/... ]
#pragma unroll
  for (int m = 0; m < 16 / R3; ++m) {
    const int j = j0 + m * T;
#pragma unroll
    for (int t = 0; t < R3; ++t) v[m * R3 + t] = sm[(j + t * (n / R3)) * SR + q];
#pragma unroll
    for (int t = 1; t < R3; ++t)
      v[m * R3 + t] = cmul(v[m * R3 + t], tw<INV>(table, (j * t) << (kTwiddleLog - LOGN)));
    if (R3 == 2) {
      const float2 a = v[m * 2];
      v[m * 2] = cadd(a, v[m * 2 + 1]);
      v[m * 2 + 1] = csub(a, v[m * 2 + 1]);
    } else if (R3 == 4) {
      dft4<INV>(v[m * 4], v[m * 4 + 1], v[m * 4 + 2], v[m * 4 + 3]);
    } else {
      dft8<INV>(v + m * 8);
    }
  }
}

template <int LOGN, int CP>
struct RegShape {
  static constexpr int n = 1 << LOGN;
  static constexpr int T = n / 16;
  static constexpr int NT = T * CP;
  static constexpr int SR = CP + 1;
};

template <int LOGN, int CP, bool INV>
__global__ void __launch_bounds__(RegShape<LOGN, CP>::NT) panel_fft_reg_kernel(const PanelArgs a) {
  using S = RegShape<LOGN, CP>;
  constexpr int n = S::n, T = S::T, SR = S::SR, R3 = n / 256;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  int j0, q;
  if (a.load_i_fastest) {
    j0 = tid % T;
    q = tid / T;
  } else {
    q = tid % CP;
    j0 = tid / CP;
  }
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const int hi = (blockIdx.x / nlo) * a.CHI + q / a.CLO;
  const int lo = (blockIdx.x % nlo) * a.CLO + q % a.CLO;
  const bool valid = hi < a.hi_total && lo < a.lo_total;
  const int b = blockIdx.y;
  const float2* __restrict__ in = a.in + (long long)b * a.in_sb + (long long)hi * a.in_shi + (long long)lo * a.in_slo;

  float2 v[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int pos = j0 + t * T;
    const int i = (pos - a.in_off) & (n - 1);
    float2 x = make_float2(0.f, 0.f);
    if (valid && i < a.nin) {
      x = __ldg(in + (long long)i * a.in_si);
      if (a.mul_i) {
        const float m = __ldg(a.mul_i + i);
        x.x *= m;
        x.y *= m;
      }
    }
    v[t] = x;
  }
  fft_core<LOGN, SR, INV>(v, sm, j0, q, a.twiddle);
  if (!valid) return;
  const float sb = a.scale * (a.mul_b ? a.mul_b[b] : 1.f);
  const long long obase = (long long)b * a.out_sb + (long long)hi * a.out_shi + (long long)lo * a.out_slo;
#pragma unroll
  for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
    for (int t = 0; t < R3; ++t) {
      const int bin = j0 + m * T + 256 * t;
      const int o = (bin - a.out_off) & (n - 1);
      if (o < a.nout) {
        float2 x = v[m * R3 + t];
        const float s = sb * (a.mul_o ? __ldg(a.mul_o + o) : 1.f);
        x.x *= s;
        x.y *= s;
        const long long off = obase + (long long)o * a.out_si;
        if (a.out_mag)
          a.out_mag[off] = sqrtf(x.x * x.x + x.y * x.y);
        else
          a.out[off] = x;
      }
    }
}

// Bluestein form: chirp the window, forward transform, multiply by bhat, inverse transform,
// chirp the kept bins.  Between the two transforms the bins are regrouped through
// shared memory into the entry layout of stage 1.
template <int LOGN, int CP>
__global__ void __launch_bounds__(RegShape<LOGN, CP>::NT) panel_bluestein_reg_kernel(
    const PanelArgs a, const float2* __restrict__ cpre, const float2* __restrict__ bhat,
    const float2* __restrict__ cpost) {
  using S = RegShape<LOGN, CP>;
  constexpr int n = S::n, T = S::T, SR = S::SR, R3 = n / 256;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int q = tid % CP, j0 = tid / CP;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const int hi = (blockIdx.x / nlo) * a.CHI + q / a.CLO;
  const int lo = (blockIdx.x % nlo) * a.CLO + q % a.CLO;
  const bool valid = hi < a.hi_total && lo < a.lo_total;
  const int b = blockIdx.y;
  const float2* __restrict__ in = a.in + (long long)b * a.in_sb + (long long)hi * a.in_shi + (long long)lo * a.in_slo;
  float2 v[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int pos = j0 + t * T;
    const int i = (pos - a.in_off) & (n - 1);
    v[t] = (valid && i < a.nin) ? cmul(__ldg(in + (long long)i * a.in_si), __ldg(cpre + i)) : make_float2(0.f, 0.f);
  }
  fft_core<LOGN, SR, false>(v, sm, j0, q, a.twiddle);
  __syncthreads();  // every thread has read its stage-3 inputs; reuse the buffer
#pragma unroll
  for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
    for (int t = 0; t < R3; ++t) {
      const int bin = j0 + m * T + 256 * t;
      sm[bin * SR + q] = cmul(v[m * R3 + t], __ldg(bhat + bin));
    }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = sm[(j0 + t * T) * SR + q];
  __syncthreads();
  fft_core<LOGN, SR, true>(v, sm, j0, q, a.twiddle);
  if (!valid) return;
  const long long obase = (long long)b * a.out_sb + (long long)hi * a.out_shi + (long long)lo * a.out_slo;
#pragma unroll
  for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
    for (int t = 0; t < R3; ++t) {
      const int bin = j0 + m * T + 256 * t;
      const int o = (bin - a.out_off) & (n - 1);
      if (o < a.nout) a.out[obase + (long long)o * a.out_si] = cmul(v[m * R3 + t], __ldg(cpost + o));
    }
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = valid ? 8 : 0;  // src-size 0 zero-fills the destination
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Persistent form: each CTA walks panels p = blockIdx.x, +gridDim.x, ... (panel =
// channel chunk + batch item).  A panel's input window is staged in shared memory by
// cp.async; once every thread has copied its 16 values into registers, the next
// panel's copy is started into the same buffer and runs under this panel's
// transform and stores.
template <int LOGN, int CP, bool INV>
__global__ void __launch_bounds__(RegShape<LOGN, CP>::NT) panel_fft_pipe_kernel(const PanelArgs a, int npanel) {
  using S = RegShape<LOGN, CP>;
  constexpr int n = S::n, T = S::T, SR = S::SR, R3 = n / 256, NT = S::NT;
  extern __shared__ float2 sm[];
  float2* xbuf = sm;            // exchange buffer [n][SR]
  float2* ibuf = sm + n * SR;   // staging [nin][CP]
  const int tid = threadIdx.x;
  int j0, q;
  if (a.load_i_fastest) {
    j0 = tid % T;
    q = tid / T;
  } else {
    q = tid % CP;
    j0 = tid / CP;
  }
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const int nchunk = ((a.hi_total + a.CHI - 1) / a.CHI) * nlo;

  // Copy work per thread: a fixed channel column and every (NT/CP)-th row (or, for
  // load_i_fastest, a fixed row residue), so each copy is a pointer increment.
  constexpr int RSTEP = NT / CP;
  auto issue = [&](int p, float2* buf) {
    const int chunk = p % nchunk, b = p / nchunk;
    const int hi0 = (chunk / nlo) * a.CHI, lo0 = (chunk % nlo) * a.CLO;
    const float2* inb = a.in + (long long)b * a.in_sb;
    if (!a.load_i_fastest) {
      const int qq = tid % CP;
      const int hi = hi0 + qq / a.CLO, lo = lo0 + qq % a.CLO;
      const bool ok = hi < a.hi_total && lo < a.lo_total;
      const float2* src = inb + (long long)hi * a.in_shi + (long long)lo * a.in_slo;
      const long long step = (long long)RSTEP * a.in_si;
      int i = tid / CP;
      src += (long long)i * a.in_si;
      for (; i < a.nin; i += RSTEP, src += step) cp_async8(buf + i * CP + qq, ok ? src : a.in, ok);
    } else {
      for (int idx = tid; idx < a.nin * CP; idx += NT) {
        const int i = idx % a.nin, qq = idx / a.nin;
        const int hi = hi0 + qq / a.CLO, lo = lo0 + qq % a.CLO;
        const bool ok = hi < a.hi_total && lo < a.lo_total;
        const float2* src = ok ? inb + (long long)i * a.in_si + (long long)hi * a.in_shi + (long long)lo * a.in_slo : a.in;
        cp_async8(buf + i * CP + qq, src, ok);
      }
    }
  };

  int p = blockIdx.x;
  if (p < npanel) issue(p, ibuf);
  cp_async_commit();
  for (; p < npanel; p += gridDim.x) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();  // the staged window is complete, and the previous panel's exchanges are done
    const int chunk = p % nchunk, b = p / nchunk;
    const int hi = (chunk / nlo) * a.CHI + q / a.CLO;
    const int lo = (chunk % nlo) * a.CLO + q % a.CLO;
    const bool valid = hi < a.hi_total && lo < a.lo_total;
    float2 v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int i = (j0 + t * T - a.in_off) & (n - 1);
      float2 x = make_float2(0.f, 0.f);
      if (i < a.nin) {
        x = ibuf[i * CP + q];
        if (a.mul_i) {
          const float m = __ldg(a.mul_i + i);
          x.x *= m;
          x.y *= m;
        }
      }
      v[t] = x;
    }
    __syncthreads();  // every thread holds its values: the buffer may be refilled
    if (p + (int)gridDim.x < npanel) issue(p + gridDim.x, ibuf);
    cp_async_commit();
    fft_core<LOGN, SR, INV>(v, xbuf, j0, q, a.twiddle);
    if (valid) {
      const float sb = a.scale * (a.mul_b ? a.mul_b[b] : 1.f);
      const long long obase = (long long)b * a.out_sb + (long long)hi * a.out_shi + (long long)lo * a.out_slo;
#pragma unroll
      for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
        for (int t = 0; t < R3; ++t) {
          const int bin = j0 + m * T + 256 * t;
          const int o = (bin - a.out_off) & (n - 1);
          if (o < a.nout) {
            float2 x = v[m * R3 + t];
            const float sc = sb * (a.mul_o ? __ldg(a.mul_o + o) : 1.f);
            x.x *= sc;
            x.y *= sc;
            const long long off = obase + (long long)o * a.out_si;
            if (a.out_mag)
              a.out_mag[off] = sqrtf(x.x * x.x + x.y * x.y);
            else
              a.out[off] = x;
          }
        }
    }
  }
}

template <class K>
cudaError_t configure(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int LOGN, int CP, bool INV>
cudaError_t launch_reg(const PanelArgs& a, cudaStream_t s) {
  using S = RegShape<LOGN, CP>;
  const int nhi = (a.hi_total + a.CHI - 1) / a.CHI;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const long long npanel = (long long)nhi * nlo * a.batch;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const size_t smem_pipe = sizeof(float2) * ((size_t)S::n * S::SR + (size_t)a.nin * CP);
  if (npanel >= 4LL * sms && smem_pipe <= 220 * 1024) {  // enough panels to stream: persistent form
    static size_t configured_pipe = 0;
    if (configured_pipe < smem_pipe) {
      cudaError_t e = configure(panel_fft_pipe_kernel<LOGN, CP, INV>, 220 * 1024);
      if (e != cudaSuccess) return e;
      configured_pipe = 220 * 1024;
    }
    const int grid = (int)std::min<long long>(npanel, (long long)sms * (smem_pipe <= 110 * 1024 ? 2 : 1));
    panel_fft_pipe_kernel<LOGN, CP, INV><<<grid, S::NT, smem_pipe, s>>>(a, (int)npanel);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(float2) * S::n * S::SR;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = configure(panel_fft_reg_kernel<LOGN, CP, INV>, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  panel_fft_reg_kernel<LOGN, CP, INV><<<dim3(nhi * nlo, a.batch), S::NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, int CP>
cudaError_t launch_bluestein_reg(const PanelArgs& a, const float2* cpre, const float2* bhat, const float2* cpost,
                                 cudaStream_t s) {
  using S = RegShape<LOGN, CP>;
  const size_t smem = sizeof(float2) * S::n * S::SR;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = configure(panel_bluestein_reg_kernel<LOGN, CP>, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int nhi = (a.hi_total + a.CHI - 1) / a.CHI;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  panel_bluestein_reg_kernel<LOGN, CP><<<dim3(nhi * nlo, a.batch), S::NT, smem, s>>>(a, cpre, bhat, cpost);
  return cudaGetLastError();
}

}  // namespace

// Panel widths of the register kernels: 512 threads per CTA.
int panel_width_reg(int logn) { return logn == 9 ? 16 : (logn == 10 ? 8 : 4); }

cudaError_t launch_panel_fft_reg(int logn, bool inverse, const PanelArgs& a, cudaStream_t s) {
  switch (logn) {
    case 9: return inverse ? launch_reg<9, 16, true>(a, s) : launch_reg<9, 16, false>(a, s);
    case 10: return inverse ? launch_reg<10, 8, true>(a, s) : launch_reg<10, 8, false>(a, s);
    case 11: return inverse ? launch_reg<11, 4, true>(a, s) : launch_reg<11, 4, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_panel_bluestein_reg(int logn, const PanelArgs& a, const float2* cpre, const float2* bhat,
                                       const float2* cpost, cudaStream_t s) {
  switch (logn) {
    case 9: return launch_bluestein_reg<9, 16>(a, cpre, bhat, cpost, s);
    case 10: return launch_bluestein_reg<10, 8>(a, cpre, bhat, cpost, s);
    case 11: return launch_bluestein_reg<11, 4>(a, cpre, bhat, cpost, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nursd
