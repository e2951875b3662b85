// Register-resident panel FFT for the long transforms (n = 512, 1024, 2048).
//
// Same contract as panel_fft_kernel (PanelArgs: a window of nin inputs placed
// at (i + in_off) mod n, nout bins kept at (o + out_off) mod n, CP channels per
// CTA), but each thread keeps 16 complex values in registers and the transform
// is three self-sorting Stockham stages of radix 16, 16 and n/256.  Data crosses
// shared memory only between stages: two exchanges per transform instead of a
// shared-memory round trip per radix-4 pass.
//
// Stage s (radix R, stride Ns) maps butterfly j: inputs x[j + t n/R],
// twiddle e^{-+2 pi i (j mod Ns) t / (Ns R)}, outputs x'[(j - j mod Ns) R + j mod Ns + t Ns].
// With T = n/16 threads per transform, thread j0 does butterfly j0 of stages 1
// and 2 and butterflies j0 + m T (m < 16/R3) of stage 3, whose outputs are the
// final bins j + 256 t.
//
// Exchange layout: element e of channel q sits at row e + PAD (e >> 4), column q
// (rows of CP values, one spare row after every 16 when CP < 16).  A half-warp
// (16 threads x 8 bytes) then hits 16 distinct bank pairs in every exchange, and
// each thread's 16 accesses are one base address plus compile-time offsets.
// Twiddles come from per-thread rows of the FFT table (two per 16-byte load).
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr float kC8 = 0.70710678118654752440f;  // cos(pi/4)
constexpr float kC16 = 0.92387953251128675613f; // cos(pi/8)
constexpr float kS16 = 0.38268343236508977173f; // sin(pi/8)

// Two-lane fp32 add and subtract in one instruction (each lane rounds as a scalar fadd would).
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " add.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

// 4-point DFT in place; the -+i rotation of the odd difference is folded into the last adds.
template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 a = padd(x0, x2), b = psub(x0, x2), c = padd(x1, x3), d = psub(x1, x3);
  x0 = padd(a, c);
  x2 = psub(a, c);
  if (INV) {  // b +- i d
    x1 = make_float2(b.x - d.y, b.y + d.x);
    x3 = make_float2(b.x + d.y, b.y - d.x);
  } else {    // b -+ i d
    x1 = make_float2(b.x + d.y, b.y - d.x);
    x3 = make_float2(b.x - d.y, b.y + d.x);
  }
}

// e^{-+2 pi i m / 16} for m = 1, 2, 3, 4, 6, 9 (constants of the regular 16-gon)
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
  v[0] = padd(e0, o0);
  v[4] = psub(e0, o0);
  v[1] = padd(e1, o1);
  v[5] = psub(e1, o1);
  v[2] = padd(e2, o2);
  v[6] = psub(e2, o2);
  v[3] = padd(e3, o3);
  v[7] = psub(e3, o3);
}

// a * w (forward) or a * conj(w) (inverse), w from the forward table.
template <bool INV>
__device__ __forceinline__ float2 twmul(float2 a, float2 w) {
  return INV ? make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y) : cmul(a, w);
}

// v[t] *= row[t] for t = 1 .. R-1, row = R consecutive table entries (16-byte aligned).
template <int R, bool INV>
__device__ __forceinline__ void twiddle_row(float2* v, const float2* __restrict__ row) {
  const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
  for (int u = 0; u < R / 2; ++u) {
    const float4 w = __ldg(r4 + u);
    if (u > 0) v[2 * u] = twmul<INV>(v[2 * u], make_float2(w.x, w.y));
    v[2 * u + 1] = twmul<INV>(v[2 * u + 1], make_float2(w.z, w.w));
  }
}

template <int LOGN, int CP>
struct RegShape {
  static constexpr int n = 1 << LOGN;
  static constexpr int T = n / 16;
  static constexpr int NT = T * CP;
  static constexpr int PAD = CP < 16 ? 1 : 0;
  static constexpr int XROWS = n + PAD * (n / 16);  // exchange buffer rows
  __device__ static int row(int e) { return e + PAD * (e >> 4); }
};

// The transform on registers v[16] of thread j0 (channel column q).
// Entry: v[t] = x[j0 + t n/16].  Exit: v[m R3 + t] = X[j0 + m T + 256 t].
template <int LOGN, int CP, bool INV>
__device__ __forceinline__ void fft_core(float2* v, float2* sm, int j0, int q, const float2* __restrict__ table) {
  using S = RegShape<LOGN, CP>;
  constexpr int n = S::n, T = S::T, R3 = n / 256, PAD = S::PAD;
  // stage 1: radix 16, Ns = 1; outputs 16 j0 + t at rows (16 + PAD) j0 + t
  dft16<INV>(v);
  {
    float2* w = sm + (16 + PAD) * j0 * CP + q;
#pragma unroll
    for (int t = 0; t < 16; ++t) w[t * (CP)] = v[t];
  }
  __syncthreads();
  // stage 2: radix 16, Ns = 16; inputs j0 + t T at rows row(j0) + t (T + PAD T/16)
  {
    const float2* r = sm + S::row(j0) * CP + q;
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = r[t * (T + PAD * (T / 16)) * CP];
  }
  twiddle_row<16, INV>(v, table + kTw2Offset + 16 * (j0 & 15));
  dft16<INV>(v);
  __syncthreads();
  {  // outputs base + 16 t, base = (j0 - k) 16 + k, at rows base + PAD (j0 - k) + t (16 + PAD)
    const int k = j0 & 15;
    float2* w = sm + ((j0 - k) * 16 + k + PAD * (j0 - k)) * CP + q;
#pragma unroll
    for (int t = 0; t < 16; ++t) w[t * (16 + PAD) * CP] = v[t];
  }
  __syncthreads();
  // stage 3: radix R3, Ns = 256, butterflies j = j0 + m T: inputs j + 256 t at rows row(j) + t (256 + 16 PAD)
#pragma unroll
  for (int m = 0; m < 16 / R3; ++m) {
    const int j = j0 + m * T;
    const float2* r = sm + S::row(j) * CP + q;
#pragma unroll
    for (int t = 0; t < R3; ++t) v[m * R3 + t] = r[t * (256 + 16 * PAD) * CP];
    twiddle_row<R3, INV>(v + m * R3, table + tw3_offset(LOGN) + j * R3);
    if (R3 == 2) {
      const float2 a = v[m * 2];
      v[m * 2] = padd(a, v[m * 2 + 1]);
      v[m * 2 + 1] = psub(a, v[m * 2 + 1]);
    } else if (R3 == 4) {
      dft4<INV>(v[m * 4], v[m * 4 + 1], v[m * 4 + 2], v[m * 4 + 3]);
    } else {
      dft8<INV>(v + m * 8);
    }
  }
}

// Stores the kept bins of thread j0: bin j0 + m T + 256 t -> output o = (bin - out_off) mod n if o < nout,
// scaled by scale * mul_b[b] * mul_o[o] (or written as a magnitude).
template <int LOGN>
__device__ __forceinline__ void store_bins(const PanelArgs& a, const float2* v, int j0, long long obase, int b) {
  constexpr int n = 1 << LOGN, T = n / 16, R3 = n / 256;
  const int opos = (j0 - a.out_off) & (n - 1);
  const int osi = (int)a.out_si;
  const float sb = a.scale * (a.mul_b ? __ldg(a.mul_b + b) : 1.f);
  if (a.out_mag) {
    float* op = a.out_mag + obase;
#pragma unroll
    for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
      for (int t = 0; t < R3; ++t) {
        const int o = (opos + m * T + 256 * t) & (n - 1);
        if (o < a.nout) {
          const float sc = sb * (a.mul_o ? __ldg(a.mul_o + o) : 1.f);
          const float2 x = make_float2(v[m * R3 + t].x * sc, v[m * R3 + t].y * sc);
          op[(long long)o * osi] = sqrtf(x.x * x.x + x.y * x.y);
        }
      }
  } else if (a.mul_o || sb != 1.f) {
    float2* op = a.out + obase;
#pragma unroll
    for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
      for (int t = 0; t < R3; ++t) {
        const int o = (opos + m * T + 256 * t) & (n - 1);
        if (o < a.nout) {
          const float sc = sb * (a.mul_o ? __ldg(a.mul_o + o) : 1.f);
          op[(long long)o * osi] = make_float2(v[m * R3 + t].x * sc, v[m * R3 + t].y * sc);
        }
      }
  } else {
    float2* op = a.out + obase;
#pragma unroll
    for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
      for (int t = 0; t < R3; ++t) {
        const int o = (opos + m * T + 256 * t) & (n - 1);
        if (o < a.nout) op[(long long)o * osi] = v[m * R3 + t];
      }
  }
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = valid ? 8 : 0;  // src-size 0 zero-fills the destination
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// One panel per CTA, inputs read from global memory straight into registers.
template <int LOGN, int CP, bool INV>
__global__ void __launch_bounds__(RegShape<LOGN, CP>::NT, 2) panel_fft_reg_kernel(const PanelArgs a) {
  using S = RegShape<LOGN, CP>;
  constexpr int n = S::n, T = S::T;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  int j0, q;
  if (a.load_i_fastest) {  // consecutive threads read consecutive inputs
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
  const int isi = (int)a.in_si;
  const int lpos = (j0 - a.in_off) & (n - 1);  // input index at FFT position j0
  float2 v[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int i = (lpos + t * T) & (n - 1);
    float2 x = make_float2(0.f, 0.f);
    if (valid && i < a.nin) {
      x = __ldg(in + (long long)i * isi);
      if (a.mul_i) {
        const float m = __ldg(a.mul_i + i);
        x.x *= m;
        x.y *= m;
      }
    }
    v[t] = x;
  }
  fft_core<LOGN, CP, INV>(v, sm, j0, q, a.twiddle);
  if (!valid) return;
  store_bins<LOGN>(a, v, j0, (long long)b * a.out_sb + (long long)hi * a.out_shi + (long long)lo * a.out_slo, b);
}

// Bluestein form: chirp the window, forward transform, multiply by bhat, inverse transform,
// chirp the kept bins.  Between the two transforms the bins are regrouped through
// shared memory into the entry layout of stage 1.
template <int LOGN, int CP>
__global__ void __launch_bounds__(RegShape<LOGN, CP>::NT) panel_bluestein_reg_kernel(
    const PanelArgs a, const float2* __restrict__ cpre, const float2* __restrict__ bhat,
    const float2* __restrict__ cpost) {
  using S = RegShape<LOGN, CP>;
  constexpr int n = S::n, T = S::T, R3 = n / 256;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int q = tid % CP, j0 = tid / CP;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const int hi = (blockIdx.x / nlo) * a.CHI + q / a.CLO;
  const int lo = (blockIdx.x % nlo) * a.CLO + q % a.CLO;
  const bool valid = hi < a.hi_total && lo < a.lo_total;
  const int b = blockIdx.y;
  const float2* __restrict__ in = a.in + (long long)b * a.in_sb + (long long)hi * a.in_shi + (long long)lo * a.in_slo;
  const int isi = (int)a.in_si, osi = (int)a.out_si;
  const int lpos = (j0 - a.in_off) & (n - 1);
  float2 v[16];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int i = (lpos + t * T) & (n - 1);
    v[t] = (valid && i < a.nin) ? cmul(__ldg(in + (long long)i * isi), __ldg(cpre + i)) : make_float2(0.f, 0.f);
  }
  fft_core<LOGN, CP, false>(v, sm, j0, q, a.twiddle);
  __syncthreads();  // every thread has read its stage-3 inputs; reuse the buffer
#pragma unroll
  for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
    for (int t = 0; t < R3; ++t) {
      const int bin = j0 + m * T + 256 * t;
      sm[S::row(bin) * CP + q] = cmul(v[m * R3 + t], __ldg(bhat + bin));
    }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < 16; ++t) v[t] = sm[S::row(j0 + t * T) * CP + q];
  __syncthreads();
  fft_core<LOGN, CP, true>(v, sm, j0, q, a.twiddle);
  if (!valid) return;
  float2* op = a.out + (long long)b * a.out_sb + (long long)hi * a.out_shi + (long long)lo * a.out_slo;
  const int opos = (j0 - a.out_off) & (n - 1);
#pragma unroll
  for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
    for (int t = 0; t < R3; ++t) {
      const int o = (opos + m * T + 256 * t) & (n - 1);
      if (o < a.nout) op[(long long)o * osi] = cmul(v[m * R3 + t], __ldg(cpost + o));
    }
}

// floor(x / d) for 0 <= x < 2^22 and d >= 1, with inv = 1.f / d: the rounded float
// quotient is within 1 of the exact one, and one correction step makes it exact.
__device__ __forceinline__ int small_div(int x, int d, float inv) {
  int qt = __float2int_rz(__int2float_rz(x) * inv);
  const int r = x - qt * d;
  qt += (r >= d) - (r < 0);
  return qt;
}

// Writes the kept bins of the panel held in xbuf as [bin][CP] (dense) to global memory:
// output o = (bin - out_off) mod n for o < nout, scaled by scale * mul_b[b] * mul_o[o]
// (or as magnitudes).  Threads take fixed channels (pairs of adjacent channels when
// vec2) and every (NT / channels)-th row, so consecutive threads store consecutive
// addresses along the contiguous channel axis.
template <int LOGN, int CP, int NT>
__device__ __forceinline__ void copy_out(const PanelArgs& a, const float2* xbuf, const float* mo, int b, int hi0,
                                         int lo0, int vec2) {
  constexpr int n = 1 << LOGN;
  const int tid = threadIdx.x;
  const float sb = a.scale * (a.mul_b ? __ldg(a.mul_b + b) : 1.f);
  const bool scaled = a.mul_o != nullptr || sb != 1.f;  // mo: shared-memory copy of mul_o[0..nout)
  const long long obase = (long long)b * a.out_sb;
  if (vec2) {  // out_slo == 1, channel pairs (qq, qq + 1) share hi and are 16-byte aligned
    constexpr int CP2 = CP / 2, RSTEP = NT / CP2;
    const int qq = 2 * (tid % CP2);
    const int hi = hi0 + qq / a.CLO, lo = lo0 + qq % a.CLO;
    if (hi >= a.hi_total || lo >= a.lo_total) return;
    const long long cbase = obase + (long long)hi * a.out_shi + lo;
    for (int o = tid / CP2; o < a.nout; o += RSTEP) {
      const int bin = (o + a.out_off) & (n - 1);
      float4 x = *reinterpret_cast<const float4*>(xbuf + bin * CP + qq);
      if (scaled) {
        const float sc = sb * (a.mul_o ? __ldg(a.mul_o + o) : 1.f);
        x.x *= sc;
        x.y *= sc;
        x.z *= sc;
        x.w *= sc;
      }
      const long long off = cbase + (long long)o * a.out_si;
      if (a.out_mag)
        *reinterpret_cast<float2*>(a.out_mag + off) =
            make_float2(sqrtf(x.x * x.x + x.y * x.y), sqrtf(x.z * x.z + x.w * x.w));
      else
        *reinterpret_cast<float4*>(a.out + off) = x;
    }
  } else {  // one channel per thread; hi fastest across threads when hi is the contiguous axis
    constexpr int RSTEP = NT / CP;
    const int c = tid % CP;
    const int qq = a.store_hi_fastest ? (c % a.CHI) * a.CLO + c / a.CHI : c;
    const int hi = hi0 + qq / a.CLO, lo = lo0 + qq % a.CLO;
    if (hi >= a.hi_total || lo >= a.lo_total) return;
    const long long cbase = obase + (long long)hi * a.out_shi + (long long)lo * a.out_slo;
    for (int o = tid / CP; o < a.nout; o += RSTEP) {
      const int bin = (o + a.out_off) & (n - 1);
      float2 x = xbuf[bin * CP + qq];
      if (scaled) {
        const float sc = sb * (a.mul_o ? __ldg(a.mul_o + o) : 1.f);
        x.x *= sc;
        x.y *= sc;
      }
      const long long off = cbase + (long long)o * a.out_si;
      if (a.out_mag)
        a.out_mag[off] = sqrtf(x.x * x.x + x.y * x.y);
      else
        a.out[off] = x;
    }
  }
}

// Persistent form: each CTA walks panels p = blockIdx.x, +gridDim.x, ... (panel p =
// batch item p / nchunk, channel chunk p mod nchunk).  A panel's input window is
// staged in shared memory ([nin][CP], followed by one all-zero row that FFT positions
// outside the window read) by cp.async; once every thread has copied its 16 values
// into registers, the next panel's copy is started into the same buffer and runs
// under this panel's transform.  The transform's bins are then written back to the
// exchange buffer in natural order and copied out row by row (copy_out).
// in_vec2 / out_vec2: the window rows (output rows) are 16-byte aligned pairs of
// channels, moved two channels at a time.
template <int LOGN, int CP, bool INV>
__global__ void __launch_bounds__(RegShape<LOGN, CP>::NT, 2) panel_fft_pipe_kernel(const PanelArgs a, int npanel,
                                                                                    int in_vec2, int out_vec2) {
  using S = RegShape<LOGN, CP>;
  constexpr int n = S::n, T = S::T, NT = S::NT, R3 = n / 256;
  extern __shared__ float2 sm[];
  float2* xbuf = sm;                   // exchange buffer [XROWS][CP]
  float2* ibuf = sm + S::XROWS * CP;   // staging [nin + 1][CP]
  const int tid = threadIdx.x;
  const int q = tid % CP, j0 = tid / CP;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const int nchunk = ((a.hi_total + a.CHI - 1) / a.CHI) * nlo;
  const float inv_nlo = 1.f / (float)nlo;
  const int qhi = q / a.CLO, qlo = q % a.CLO;
  // copy roles: channel pair cq2, cq2 + 1 (in_vec2) or channel q, of rows crow + k RSTEP
  const int cq2 = 2 * (tid % (CP / 2));
  const int cq2hi = cq2 / a.CLO, cq2lo = cq2 % a.CLO;
  if (tid < CP) ibuf[a.nin * CP + tid] = make_float2(0.f, 0.f);  // the zero row
  float* mo = reinterpret_cast<float*>(ibuf + (a.nin + 1) * CP);  // mul_o[0..nout), if any
  if (a.mul_o)
    for (int o = tid; o < a.nout; o += NT) mo[o] = __ldg(a.mul_o + o);

  auto issue = [&](int b, int chunk) {
    const int hc = small_div(chunk, nlo, inv_nlo);
    const int hi0 = hc * a.CHI, lo0 = (chunk - hc * nlo) * a.CLO;
    const float2* inb = a.in + (long long)b * a.in_sb;
    if (a.load_i_fastest) {  // the axis is contiguous in memory: consecutive threads copy consecutive i
      for (int idx = tid; idx < a.nin * CP; idx += NT) {
        const int i = idx % a.nin, qq = idx / a.nin;
        const int hi = hi0 + qq / a.CLO, lo = lo0 + qq % a.CLO;
        const bool ok = hi < a.hi_total && lo < a.lo_total;
        const float2* src = ok ? inb + (long long)i * a.in_si + (long long)hi * a.in_shi + (long long)lo * a.in_slo : a.in;
        cp_async8(ibuf + i * CP + qq, src, ok);
      }
    } else if (in_vec2) {
      constexpr int RSTEP = NT / (CP / 2);
      const int hi = hi0 + cq2hi, lo = lo0 + cq2lo;
      const bool ok = hi < a.hi_total && lo < a.lo_total;
      int i = tid / (CP / 2);
      const float2* src = inb + (long long)hi * a.in_shi + lo + (long long)i * a.in_si;
      const long long step = (long long)RSTEP * a.in_si;
      for (; i < a.nin; i += RSTEP, src += step) cp_async16(ibuf + i * CP + cq2, ok ? src : a.in, ok);
    } else {
      constexpr int RSTEP = NT / CP;
      const int hi = hi0 + qhi, lo = lo0 + qlo;
      const bool ok = hi < a.hi_total && lo < a.lo_total;
      int i = tid / CP;
      const float2* src = inb + (long long)hi * a.in_shi + (long long)lo * a.in_slo + (long long)i * a.in_si;
      const long long step = (long long)RSTEP * a.in_si;
      for (; i < a.nin; i += RSTEP, src += step) cp_async8(ibuf + i * CP + q, ok ? src : a.in, ok);
    }
  };

  const int lpos = (j0 - a.in_off) & (n - 1);  // input index at FFT position j0
  const float2* rq = ibuf + q;
  const int step_b = gridDim.x / nchunk, step_c = gridDim.x % nchunk;
  int p = blockIdx.x;
  int cb = p / nchunk, cc = p % nchunk;  // batch item and chunk of panel p
  if (p < npanel) issue(cb, cc);
  cp_async_commit();
  for (; p < npanel; p += gridDim.x) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();  // the staged window is complete, and the previous panel's copy-out is done
    const int hc = small_div(cc, nlo, inv_nlo);
    const int hi0 = hc * a.CHI, lo0 = (cc - hc * nlo) * a.CLO;
    const int b = cb;
    float2 v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = rq[min((lpos + t * T) & (n - 1), a.nin) * CP];
    if (a.mul_i) {
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int i = (lpos + t * T) & (n - 1);
        if (i < a.nin) {
          const float m = __ldg(a.mul_i + i);
          v[t].x *= m;
          v[t].y *= m;
        }
      }
    }
    __syncthreads();  // every thread holds its values: the buffer may be refilled
    cb += step_b;
    cc += step_c;
    if (cc >= nchunk) {
      cc -= nchunk;
      ++cb;
    }
    if (p + (int)gridDim.x < npanel) issue(cb, cc);
    cp_async_commit();
    fft_core<LOGN, CP, INV>(v, xbuf, j0, q, a.twiddle);
    __syncthreads();  // every thread has read its last-stage inputs
    {
      float2* w = xbuf + j0 * CP + q;
#pragma unroll
      for (int m = 0; m < 16 / R3; ++m)
#pragma unroll
        for (int t = 0; t < R3; ++t) w[(m * T + 256 * t) * CP] = v[m * R3 + t];
    }
    __syncthreads();
    copy_out<LOGN, CP, NT>(a, xbuf, mo, b, hi0, lo0, out_vec2);
  }
}

// Copies panel (b, chunk)'s input window into the staging buffer [nin][CP] with cp.async
// (the caller commits): two channels per 16-byte copy when in_vec2, one per 8-byte copy
// otherwise, or consecutive rows per thread when the axis is contiguous in memory.
template <int CP, int NT>
struct WindowStager {
  const PanelArgs& a;
  float2* ibuf;
  int tid, nlo, in_vec2;
  float inv_nlo;
  __device__ __forceinline__ void operator()(int b, int chunk) const {
    const int q = tid % CP, cq2 = 2 * (tid % (CP / 2));
    const int hc = small_div(chunk, nlo, inv_nlo);
    const int hi0 = hc * a.CHI, lo0 = (chunk - hc * nlo) * a.CLO;
    const float2* inb = a.in + (long long)b * a.in_sb;
    if (a.load_i_fastest) {
      for (int idx = tid; idx < a.nin * CP; idx += NT) {
        const int i = idx % a.nin, qq = idx / a.nin;
        const int hi = hi0 + qq / a.CLO, lo = lo0 + qq % a.CLO;
        const bool ok = hi < a.hi_total && lo < a.lo_total;
        const float2* src = ok ? inb + (long long)i * a.in_si + (long long)hi * a.in_shi + (long long)lo * a.in_slo : a.in;
        cp_async8(ibuf + i * CP + qq, src, ok);
      }
    } else if (in_vec2) {
      constexpr int RSTEP = NT / (CP / 2);
      const int hi = hi0 + cq2 / a.CLO, lo = lo0 + cq2 % a.CLO;
      const bool ok = hi < a.hi_total && lo < a.lo_total;
      int i = tid / (CP / 2);
      const float2* src = inb + (long long)hi * a.in_shi + lo + (long long)i * a.in_si;
      const long long step = (long long)RSTEP * a.in_si;
      for (; i < a.nin; i += RSTEP, src += step) cp_async16(ibuf + i * CP + cq2, ok ? src : a.in, ok);
    } else {
      constexpr int RSTEP = NT / CP;
      const int hi = hi0 + q / a.CLO, lo = lo0 + q % a.CLO;
      const bool ok = hi < a.hi_total && lo < a.lo_total;
      int i = tid / CP;
      const float2* src = inb + (long long)hi * a.in_shi + (long long)lo * a.in_slo + (long long)i * a.in_si;
      const long long step = (long long)RSTEP * a.in_si;
      for (; i < a.nin; i += RSTEP, src += step) cp_async8(ibuf + i * CP + q, ok ? src : a.in, ok);
    }
  }
};

// Stages panel (b, chunk)'s transfer products (PanelArgs::prod_g) instead of a plain window: per
// window row i, the two spectrum values U[b][i][f0..f0+1] and the table rows of those two
// frequencies for the four depths, five 16-byte copies into a row of kProdRow values
// [u0, u1, g(0, 0..3), g(1, 0..3)] (the caller commits).
constexpr int kProdRow = 10;
// Batch order of the product-staging pass: item j is mode row ky = 0, 1, -1, 2, -2, ..., then -M/2
// (stored at b = ky + M/2), so the rows +ky and -ky, which use the same table classes, run back
// to back and the second finds the classes in L2.
__device__ __forceinline__ int prod_row(int j, int M) {
  if (j == M - 1) return 0;
  const int m = (j + 1) >> 1;
  return M / 2 + ((j & 1) ? m : -m);
}
template <int NT>
struct ProductStager {
  const PanelArgs& a;
  float2* ibuf;
  int tid;
  __device__ __forceinline__ void operator()(int b, int chunk) const {
    const int M = a.nin, f0 = 2 * chunk, ay = abs(b - M / 2);
    const float2* ub = a.in + (long long)b * a.in_sb + f0;
    for (int idx = tid; idx < M * 5; idx += NT) {
      const int i = idx / 5, part = idx - 5 * i;
      float2* dst = ibuf + i * kProdRow;
      if (part == 0) {
        cp_async16(dst, ub + (long long)i * a.in_si, true);
      } else {
        const int ax = abs(i - M / 2), p = max(ax, ay), q = min(ax, ay);
        const int j = (part - 1) >> 1, h = (part - 1) & 1;
        const float2* g = a.prod_g + ((long long)(p * (p + 1) / 2 + q) * a.prod_F + f0 + j) * a.prod_Z + a.prod_z0 + 2 * h;
        cp_async16(dst + 2 + 4 * j + 2 * h, g, true);
      }
    }
  }
};

// ------------------------------------------------------------------ radix-32 form
// For n = 512, 1024: two Stockham stages, radix 32 then R2 = n / 32.  T = n / 32 threads per
// transform, 32 values each.  Stage 1: thread j0 < T does butterfly j0 (a 32-point DFT of
// x[j0 + T t]) and writes x'[32 j0 + k].  Stage 2: butterflies j < 32 (32 / R2 per thread,
// j = j0 + T m) read x'[j + 32 t], t < R2, twiddle W_n^{j t}, and give X[j + 32 k].  One
// exchange; element e sits at row e + PADX (e >> 5) (a spare row after every 32 when a
// half-warp spans two rows), so both exchange directions are conflict-free.

constexpr float kW32C1 = 0.98078528040323044913f, kW32S1 = 0.19509032201612826785f;
constexpr float kW32C2 = 0.92387953251128675613f, kW32S2 = 0.38268343236508977173f;
constexpr float kW32C3 = 0.83146961230254523708f, kW32S3 = 0.55557023301960222474f;
constexpr float kW32C4 = 0.70710678118654752440f;

// a * W32^{-+m} (forward e^{-2 pi i m / 32}, inverse e^{+2 pi i m / 32}) for a constant m < 32.
template <bool INV, int M>
__device__ __forceinline__ float2 rot32(float2 a) {
  constexpr int m = M & 31;
  if (m == 0) return a;
  if (m == 8) return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  if (m == 16) return make_float2(-a.x, -a.y);
  if (m == 24) return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
  // cos and sin of 2 pi m / 32 from the first octant
  constexpr int o = m & 7, q = m >> 3;
  constexpr float c0 = o == 0 ? 1.f : o == 1 ? kW32C1 : o == 2 ? kW32C2 : o == 3 ? kW32C3 : o == 4 ? kW32C4
                       : o == 5 ? kW32S3 : o == 6 ? kW32S2 : kW32S1;
  constexpr float s0 = o == 0 ? 0.f : o == 1 ? kW32S1 : o == 2 ? kW32S2 : o == 3 ? kW32S3 : o == 4 ? kW32C4
                       : o == 5 ? kW32C3 : o == 6 ? kW32C2 : kW32C1;
  // rotate the octant angle by q quarter turns: (c, s) -> (-s, c)
  constexpr float c = q == 0 ? c0 : q == 1 ? -s0 : q == 2 ? -c0 : s0;
  constexpr float sn = q == 0 ? s0 : q == 1 ? c0 : q == 2 ? -s0 : -c0;
  return cmul(a, make_float2(c, INV ? sn : -sn));
}

template <bool INV, int N1, int K2>
__device__ __forceinline__ void rot32_at(float2* y) { y[N1 * 8 + K2] = rot32<INV, N1 * K2>(y[N1 * 8 + K2]); }

// In-place 32-point DFT: out[8 k1 + k2] = sum_n x[n] W32^{n k}, via 8-point DFTs over n2 of
// x[n1 + 4 n2], twiddles W32^{n1 k2}, and 4-point DFTs over n1.
template <bool INV>
__device__ __forceinline__ void dft32(float2* v) {
  float2 y[32];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    float2 t[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) t[n2] = v[n1 + 4 * n2];
    dft8<INV>(t);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) y[n1 * 8 + k2] = t[k2];
  }
  rot32_at<INV, 1, 1>(y); rot32_at<INV, 1, 2>(y); rot32_at<INV, 1, 3>(y); rot32_at<INV, 1, 4>(y);
  rot32_at<INV, 1, 5>(y); rot32_at<INV, 1, 6>(y); rot32_at<INV, 1, 7>(y);
  rot32_at<INV, 2, 1>(y); rot32_at<INV, 2, 2>(y); rot32_at<INV, 2, 3>(y); rot32_at<INV, 2, 4>(y);
  rot32_at<INV, 2, 5>(y); rot32_at<INV, 2, 6>(y); rot32_at<INV, 2, 7>(y);
  rot32_at<INV, 3, 1>(y); rot32_at<INV, 3, 2>(y); rot32_at<INV, 3, 3>(y); rot32_at<INV, 3, 4>(y);
  rot32_at<INV, 3, 5>(y); rot32_at<INV, 3, 6>(y); rot32_at<INV, 3, 7>(y);
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) {
    float2 a = y[k2], b = y[8 + k2], c = y[16 + k2], d = y[24 + k2];
    dft4<INV>(a, b, c, d);
    v[k2] = a;
    v[8 + k2] = b;
    v[16 + k2] = c;
    v[24 + k2] = d;
  }
}

template <int LOGN, int CP>
struct R32Shape {
  static constexpr int n = 1 << LOGN;
  static constexpr int T = n / 32;        // threads per transform
  static constexpr int R2 = n / 32;       // radix of the second stage
  static constexpr int NT = T * CP;
  static constexpr int PADX = (CP < 16) ? 1 : 0;
  static constexpr int XROWS = n + PADX * (n / 32);
};

// The two radix-32 stages on v[32] (thread j0, channel column q): entry v[t] = x[j0 + T t],
// exit v[m R2 + k] = X[j0 + T m + 32 k].  after_exchange() runs right after the exchange
// barrier (every thread has finished its stage-1 work).
template <int LOGN, int CP, bool INV, class Hook>
__device__ __forceinline__ void fft32_core(float2* v, float2* xbuf, int j0, int q, const float2* __restrict__ tw2,
                                           Hook&& after_exchange) {
  using S = R32Shape<LOGN, CP>;
  constexpr int T = S::T, R2 = S::R2, PADX = S::PADX;
  // stage 1: outputs 32 j0 + k at rows 32 j0 + k + PADX j0
  dft32<INV>(v);
  {
    float2* w = xbuf + (32 + PADX) * j0 * CP + q;
#pragma unroll
    for (int k = 0; k < 32; ++k) w[k * CP] = v[k];
  }
  __syncthreads();
  after_exchange();
  // stage 2: butterflies j = j0 + T m read rows j + (32 + PADX) t
#pragma unroll
  for (int m = 0; m < 32 / R2; ++m) {
    const int j = j0 + T * m;
    const float2* r = xbuf + j * CP + q;
#pragma unroll
    for (int t = 0; t < R2; ++t) v[m * R2 + t] = r[t * (32 + PADX) * CP];
    twiddle_row<R2, INV>(v + m * R2, tw2 + j * R2);
    if constexpr (R2 == 32)
      dft32<INV>(v + m * R2);
    else if constexpr (R2 == 16)
      dft16<INV>(v + m * R2);
    else
      dft8<INV>(v + m * R2);
  }
}

// Bins of v (fft32_core exit order) -> xbuf rows in natural order, [n][CP].
template <int LOGN, int CP>
__device__ __forceinline__ void store_bins32(const float2* v, float2* xbuf, int j0, int q) {
  using S = R32Shape<LOGN, CP>;
  float2* w = xbuf + j0 * CP + q;
#pragma unroll
  for (int m = 0; m < 32 / S::R2; ++m)
#pragma unroll
    for (int k = 0; k < S::R2; ++k) w[(S::T * m + 32 * k) * CP] = v[m * S::R2 + k];
}

// Kept bins of fft32_core's exit registers straight to global memory (direct form of the copy-out:
// one channel per panel column, channels contiguous, no magnitude): bin j0 + T m + 32 k of channel q
// -> output o = (bin - out_off) mod n if o < nout, scaled by scale * mul_b[b] * mo[o].  A warp's store
// covers 4 bins x 8 channels, four 64-byte runs, as the shared-memory copy-out's rows do.
template <int LOGN, int CP>
__device__ __forceinline__ void store_direct32(const PanelArgs& a, const float2* v, const float* mo, int b, int hi0,
                                               int lo0, int j0, int q) {
  using S = R32Shape<LOGN, CP>;
  constexpr int n = S::n;
  const int lo = lo0 + q;
  if (hi0 >= a.hi_total || lo >= a.lo_total) return;
  const float sb = a.scale * (a.mul_b ? __ldg(a.mul_b + b) : 1.f);
  const bool scaled = a.mul_o != nullptr || sb != 1.f;
  float2* base = a.out + (long long)b * a.out_sb + (long long)hi0 * a.out_shi + lo;
#pragma unroll
  for (int m = 0; m < 32 / S::R2; ++m)
#pragma unroll
    for (int k = 0; k < S::R2; ++k) {
      const int o = (j0 + S::T * m + 32 * k - a.out_off) & (n - 1);
      if (o < a.nout) {
        float2 x = v[m * S::R2 + k];
        if (scaled) {
          const float sc = a.mul_o ? sb * mo[o] : sb;
          x.x *= sc;
          x.y *= sc;
        }
        base[(long long)o * a.out_si] = x;
      }
    }
}

// Persistent radix-32 form: same panels, staging, zero row and copy-out as
// panel_fft_pipe_kernel; four CTA barriers per panel, two when the bins are stored directly
// (direct: see store_direct32).
// PROD: the window holds transfer products staged by ProductStager (CP = 8).
template <int LOGN, int CP, bool INV, bool PROD = false>
__global__ void __launch_bounds__(R32Shape<LOGN, CP>::NT, R32Shape<LOGN, CP>::NT >= 256 ? 2 : 3) panel_fft32_kernel(
    const PanelArgs a, int npanel, int in_vec2, int out_vec2, int direct) {
  pdl_wait();  // the input comes from the kernel before (and the output may be what it read)
  pdl_trigger();
  using S = R32Shape<LOGN, CP>;
  constexpr int n = S::n, T = S::T, NT = S::NT;
  constexpr int RS = PROD ? kProdRow : CP;  // staging row length
  static_assert(!PROD || CP == 8, "transfer products are staged for 8-channel panels");
  extern __shared__ float2 sm[];
  float2* xbuf = sm;                   // exchange buffer [XROWS][CP], then the bins [n][CP]
  float2* ibuf = sm + S::XROWS * CP;   // staging [nin + 1][RS]
  const int tid = threadIdx.x;
  const int q = tid % CP, j0 = tid / CP;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const int nchunk = ((a.hi_total + a.CHI - 1) / a.CHI) * nlo;
  const float inv_nlo = 1.f / (float)nlo;
  if (tid < RS) ibuf[a.nin * RS + tid] = make_float2(0.f, 0.f);  // the zero row
  float* mo = reinterpret_cast<float*>(ibuf + (a.nin + 1) * RS);  // mul_o[0..nout), if any
  if (a.mul_o)
    for (int o = tid; o < a.nout; o += NT) mo[o] = __ldg(a.mul_o + o);
  auto issue = [&](int b, int chunk) {
    if constexpr (PROD)
      ProductStager<NT>{a, ibuf, tid}(prod_row(b, a.nin), chunk);
    else
      WindowStager<CP, NT>{a, ibuf, tid, nlo, in_vec2, inv_nlo}(b, chunk);
  };

  const int lpos = (j0 - a.in_off) & (n - 1);  // input index at FFT position j0
  const float2* rq = ibuf + q;
  const float2* __restrict__ tw2 = a.twiddle + tw32_offset(LOGN);
  const int step_b = gridDim.x / nchunk, step_c = gridDim.x % nchunk;
  int p = blockIdx.x;
  int cb = p / nchunk, cc = p % nchunk;
  if (p < npanel) issue(cb, cc);
  cp_async_commit();
  for (; p < npanel; p += gridDim.x) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();  // the staged window is complete, and the previous panel's copy-out is done
    const int hc = small_div(cc, nlo, inv_nlo);
    const int hi0 = hc * a.CHI, lo0 = (cc - hc * nlo) * a.CLO;
    const int b = PROD ? prod_row(cb, a.nin) : cb;
    float2 v[32];
    if constexpr (PROD) {  // u * g of the staged row: u of frequency q / 4, g of channel q
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const float2* row = ibuf + min((lpos + t * T) & (n - 1), a.nin) * RS;
        v[t] = cmul(row[q >> 2], row[2 + q]);
      }
    } else {
#pragma unroll
      for (int t = 0; t < 32; ++t) v[t] = rq[min((lpos + t * T) & (n - 1), a.nin) * CP];
    }
    if (a.mul_i) {
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int i = (lpos + t * T) & (n - 1);
        if (i < a.nin) {
          const float m = __ldg(a.mul_i + i);
          v[t].x *= m;
          v[t].y *= m;
        }
      }
    }
    __syncthreads();  // every thread holds its window: start the next panel's copy now, so it has
                      // the whole transform to land
    cb += step_b;
    cc += step_c;
    if (cc >= nchunk) {
      cc -= nchunk;
      ++cb;
    }
    if (p + (int)gridDim.x < npanel) issue(cb, cc);
    cp_async_commit();
    fft32_core<LOGN, CP, INV>(v, xbuf, j0, q, tw2, [] {});
    if (direct) {  // the next panel's first exchange writes follow two CTA barriers
      store_direct32<LOGN, CP>(a, v, mo, b, hi0, lo0, j0, q);
      continue;
    }
    __syncthreads();  // every thread has read its stage-2 inputs
    store_bins32<LOGN, CP>(v, xbuf, j0, q);
    __syncthreads();
    copy_out<LOGN, CP, NT>(a, xbuf, mo, b, hi0, lo0, out_vec2);
  }
}

// Persistent Bluestein form for n = 512, 1024: the staged window times cpre, the forward
// transform, times bhat, regrouped through shared memory into the entry order, the inverse
// transform, and the kept bins times cpost, copied out row by row.
template <int LOGN, int CP>
__global__ void __launch_bounds__(R32Shape<LOGN, CP>::NT, R32Shape<LOGN, CP>::NT >= 256 ? 2 : 3)
    panel_bluestein32_kernel(const PanelArgs a, int npanel, int in_vec2, int out_vec2,
                             const float2* __restrict__ cpre, const float2* __restrict__ bhat,
                             const float2* __restrict__ cpost) {
  using S = R32Shape<LOGN, CP>;
  constexpr int n = S::n, T = S::T, NT = S::NT, R2 = S::R2;
  extern __shared__ float2 sm[];
  float2* xbuf = sm;
  float2* ibuf = sm + S::XROWS * CP;
  const int tid = threadIdx.x;
  const int q = tid % CP, j0 = tid / CP;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const int nchunk = ((a.hi_total + a.CHI - 1) / a.CHI) * nlo;
  const float inv_nlo = 1.f / (float)nlo;
  if (tid < CP) ibuf[a.nin * CP + tid] = make_float2(0.f, 0.f);  // the zero row
  const WindowStager<CP, NT> issue{a, ibuf, tid, nlo, in_vec2, inv_nlo};
  const int lpos = (j0 - a.in_off) & (n - 1);
  const float2* rq = ibuf + q;
  const float2* __restrict__ tw2 = a.twiddle + tw32_offset(LOGN);
  const int step_b = gridDim.x / nchunk, step_c = gridDim.x % nchunk;
  int p = blockIdx.x;
  int cb = p / nchunk, cc = p % nchunk;
  if (p < npanel) issue(cb, cc);
  cp_async_commit();
  for (; p < npanel; p += gridDim.x) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int b = cb, c_cur = cc;
    float2 v[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = rq[min((lpos + t * T) & (n - 1), a.nin) * CP];  // zero row outside
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = cmul(v[t], __ldg(cpre + min((lpos + t * T) & (n - 1), a.nin - 1)));
    __syncthreads();  // every thread holds its window: start the next panel's copy
    cb += step_b;
    cc += step_c;
    if (cc >= nchunk) {
      cc -= nchunk;
      ++cb;
    }
    if (p + (int)gridDim.x < npanel) issue(cb, cc);
    cp_async_commit();
    fft32_core<LOGN, CP, false>(v, xbuf, j0, q, tw2, [] {});
#pragma unroll
    for (int m = 0; m < 32 / R2; ++m)
#pragma unroll
      for (int k = 0; k < R2; ++k) v[m * R2 + k] = cmul(v[m * R2 + k], __ldg(bhat + j0 + T * m + 32 * k));
    __syncthreads();
    store_bins32<LOGN, CP>(v, xbuf, j0, q);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = xbuf[(j0 + T * t) * CP + q];
    __syncthreads();
    fft32_core<LOGN, CP, true>(v, xbuf, j0, q, tw2, [] {});
    __syncthreads();
    store_bins32<LOGN, CP>(v, xbuf, j0, q);
    __syncthreads();
    // kept bins times cpost[o]
    const int hc = small_div(c_cur, nlo, inv_nlo);
    const int hi0 = hc * a.CHI, lo0 = (c_cur - hc * nlo) * a.CLO;
    const long long obase = (long long)b * a.out_sb;
    if (out_vec2) {
      constexpr int CP2 = CP / 2, RSTEP = NT / CP2;
      const int qq = 2 * (tid % CP2);
      const int hi = hi0 + qq / a.CLO, lo = lo0 + qq % a.CLO;
      if (hi < a.hi_total && lo < a.lo_total) {
        const long long cbase = obase + (long long)hi * a.out_shi + lo;
        for (int o = tid / CP2; o < a.nout; o += RSTEP) {
          const int bin = (o + a.out_off) & (n - 1);
          const float4 x = *reinterpret_cast<const float4*>(xbuf + bin * CP + qq);
          const float2 c = __ldg(cpost + o);
          const float2 y0 = cmul(make_float2(x.x, x.y), c), y1 = cmul(make_float2(x.z, x.w), c);
          *reinterpret_cast<float4*>(a.out + cbase + (long long)o * a.out_si) = make_float4(y0.x, y0.y, y1.x, y1.y);
        }
      }
    } else {
      constexpr int RSTEP = NT / CP;
      const int hi = hi0 + q / a.CLO, lo = lo0 + q % a.CLO;
      if (hi < a.hi_total && lo < a.lo_total) {
        const long long cbase = obase + (long long)hi * a.out_shi + (long long)lo * a.out_slo;
        for (int o = tid / CP; o < a.nout; o += RSTEP) {
          const int bin = (o + a.out_off) & (n - 1);
          a.out[cbase + (long long)o * a.out_si] = cmul(xbuf[bin * CP + q], __ldg(cpost + o));
        }
      }
    }
  }
}

template <class K>
cudaError_t configure(K kernel, size_t smem) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  return sms;
}

// Element offsets along the axis are 32-bit in the kernels: n * stride must fit.
bool axis_offsets_fit(int n, const PanelArgs& a) {
  const long long lim = 1LL << 31;
  return a.in_si >= 0 && a.out_si >= 0 && (long long)n * a.in_si < lim && (long long)n * a.out_si < lim;
}

template <int LOGN, int CP, bool INV>
cudaError_t launch_reg(const PanelArgs& a, cudaStream_t s) {
  using S = RegShape<LOGN, CP>;
  if (!axis_offsets_fit(S::n, a)) return cudaErrorInvalidValue;
  const int nhi = (a.hi_total + a.CHI - 1) / a.CHI;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const long long npanel = (long long)nhi * nlo * a.batch;
  const int sms = sm_count();
  const size_t xbytes = sizeof(float2) * (size_t)S::XROWS * CP;
  const size_t mo_bytes = a.mul_o ? sizeof(float) * (size_t)a.nout : 0;  // shared copy of mul_o
  const size_t smem_pipe = xbytes + sizeof(float2) * (size_t)(a.nin + 1) * CP + mo_bytes;
  const void* optr = a.out_mag ? static_cast<const void*>(a.out_mag) : static_cast<const void*>(a.out);
  const int in_vec2 = !a.load_i_fastest && a.in_slo == 1 && a.CLO % 2 == 0 && a.lo_total % 2 == 0 &&
                      reinterpret_cast<uintptr_t>(a.in) % 16 == 0 && a.in_sb % 2 == 0 && a.in_si % 2 == 0 &&
                      a.in_shi % 2 == 0;
  const int out_vec2 = a.out_slo == 1 && a.CLO % 2 == 0 && a.lo_total % 2 == 0 &&
                       reinterpret_cast<uintptr_t>(optr) % (a.out_mag ? 8 : 16) == 0 && a.out_sb % 2 == 0 &&
                       a.out_si % 2 == 0 && a.out_shi % 2 == 0;
  if (a.prod_g) {  // transfer products on load: the radix-32 persistent form only
    if constexpr ((LOGN == 9 || LOGN == 10) && CP == 8) {
      using R = R32Shape<LOGN, CP>;
      if (a.CHI != 1 || a.hi_total != 1 || a.lo_total % CP != 0 || a.prod_F % 2 != 0 || a.prod_Z % 4 != 0 ||
          a.prod_z0 % 4 != 0 || a.nin != S::n || a.batch != a.nin || a.in_slo != 1 || a.mul_i || a.mul_o)
        return cudaErrorInvalidValue;
      const size_t smemp = sizeof(float2) * ((size_t)R::XROWS * CP + (size_t)(a.nin + 1) * kProdRow);
      auto kern = panel_fft32_kernel<LOGN, CP, INV, true>;
      static bool configured_p = false;
      static int occ_p = 1;
      if (!configured_p) {
        cudaError_t e = configure(kern, 220 * 1024);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, R::NT, smemp);
        if (e != cudaSuccess) return e;
        occ_p = std::max(nb, 1);
        configured_p = true;
      }
      const int grid = (int)std::min<long long>(npanel, (long long)sms * occ_p);
      kern<<<grid, R::NT, smemp, s>>>(a, (int)npanel, 0, out_vec2, 0);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if constexpr (LOGN == 9 || LOGN == 10) {  // radix-32 persistent form
    using R = R32Shape<LOGN, CP>;
    const size_t smem32 = sizeof(float2) * ((size_t)R::XROWS * CP + (size_t)(a.nin + 1) * CP) + mo_bytes;
    if (npanel >= 4LL * sms && smem32 <= 220 * 1024 && (long long)nhi * nlo < (1LL << 22)) {
      auto kern = panel_fft32_kernel<LOGN, CP, INV>;
      static bool configured32 = false;
      static size_t occ_smem32 = 0;
      static int occ32 = 1;
      if (!configured32) {
        cudaError_t e = configure(kern, 220 * 1024);
        if (e != cudaSuccess) return e;
        configured32 = true;
      }
      if (occ_smem32 != smem32) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, R::NT, smem32);
        if (e != cudaSuccess) return e;
        occ32 = std::max(nb, 1);
        occ_smem32 = smem32;
      }
      const int grid = (int)std::min<long long>(npanel, (long long)sms * occ32);
      // bins straight from registers where a panel column is one contiguous channel (fine FFT x and y:
      // 0.154 and 0.168 ms vs 0.158 and 0.183 ms through the shared-memory copy-out)
      const int direct = !a.out_mag && a.CHI == 1 && a.CLO == CP && a.out_slo == 1 && !a.store_hi_fastest;
      return launch_pdl(kern, dim3(grid), dim3(R::NT), smem32, s, a, (int)npanel, in_vec2, out_vec2, direct);
    }
  }
  if (npanel >= 4LL * sms && smem_pipe <= 220 * 1024 && (long long)nhi * nlo < (1LL << 22)) {  // persistent form
    auto kern = panel_fft_pipe_kernel<LOGN, CP, INV>;
    static bool configured = false;
    static size_t occ_smem = 0;
    static int occ = 1;
    if (!configured) {
      cudaError_t e = configure(kern, 220 * 1024);
      if (e != cudaSuccess) return e;
      configured = true;
    }
    if (occ_smem != smem_pipe) {
      int nb = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, S::NT, smem_pipe);
      if (e != cudaSuccess) return e;
      occ = std::max(nb, 1);
      occ_smem = smem_pipe;
    }
    const int grid = (int)std::min<long long>(npanel, (long long)sms * occ);
    kern<<<grid, S::NT, smem_pipe, s>>>(a, (int)npanel, in_vec2, out_vec2);
    return cudaGetLastError();
  }
  static bool configured = false;
  if (!configured) {
    cudaError_t e = configure(panel_fft_reg_kernel<LOGN, CP, INV>, xbytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  panel_fft_reg_kernel<LOGN, CP, INV><<<dim3(nhi * nlo, a.batch), S::NT, xbytes, s>>>(a);
  return cudaGetLastError();
}

template <int LOGN, int CP>
cudaError_t launch_bluestein_reg(const PanelArgs& a, const float2* cpre, const float2* bhat, const float2* cpost,
                                 cudaStream_t s) {
  using S = RegShape<LOGN, CP>;
  if (!axis_offsets_fit(S::n, a)) return cudaErrorInvalidValue;
  if constexpr (LOGN == 9 || LOGN == 10) {  // radix-32 persistent form
    using R = R32Shape<LOGN, CP>;
    const int nhi = (a.hi_total + a.CHI - 1) / a.CHI;
    const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
    const long long npanel = (long long)nhi * nlo * a.batch;
    const int sms = sm_count();
    const size_t smem32 = sizeof(float2) * ((size_t)R::XROWS * CP + (size_t)(a.nin + 1) * CP);
    if (npanel >= 4LL * sms && smem32 <= 220 * 1024 && (long long)nhi * nlo < (1LL << 22) && a.nin >= 1 &&
        !a.load_i_fastest) {
      auto kern = panel_bluestein32_kernel<LOGN, CP>;
      static bool configured32 = false;
      static size_t occ_smem32 = 0;
      static int occ32 = 1;
      if (!configured32) {
        cudaError_t e = configure(kern, 220 * 1024);
        if (e != cudaSuccess) return e;
        configured32 = true;
      }
      if (occ_smem32 != smem32) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, R::NT, smem32);
        if (e != cudaSuccess) return e;
        occ32 = std::max(nb, 1);
        occ_smem32 = smem32;
      }
      const int in_vec2 = a.in_slo == 1 && a.CLO % 2 == 0 && a.lo_total % 2 == 0 &&
                          reinterpret_cast<uintptr_t>(a.in) % 16 == 0 && a.in_sb % 2 == 0 && a.in_si % 2 == 0 &&
                          a.in_shi % 2 == 0;
      const int out_vec2 = a.out_slo == 1 && a.CLO % 2 == 0 && a.lo_total % 2 == 0 &&
                           reinterpret_cast<uintptr_t>(a.out) % 16 == 0 && a.out_sb % 2 == 0 && a.out_si % 2 == 0 &&
                           a.out_shi % 2 == 0;
      const int grid = (int)std::min<long long>(npanel, (long long)sms * occ32);
      kern<<<grid, R::NT, smem32, s>>>(a, (int)npanel, in_vec2, out_vec2, cpre, bhat, cpost);
      return cudaGetLastError();
    }
  }
  const size_t smem = sizeof(float2) * (size_t)S::XROWS * CP;
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

// Panel widths (channels per CTA) of the register kernels.
int panel_width_reg(int logn) { return logn == 11 ? 4 : 8; }

// n = 256 as 32 x 8 in the radix-32 persistent form, 16-channel panels (the width of the shared-memory
// form it replaces); cudaErrorNotSupported when the launch is too small for a persistent grid.
cudaError_t launch_panel_fft32_256(bool inverse, const PanelArgs& a, cudaStream_t s) {
  constexpr int LOGN = 8, CP = 16;
  using R = R32Shape<LOGN, CP>;
  if (a.CHI * a.CLO != CP || a.prod_g || !axis_offsets_fit(R::n, a)) return cudaErrorNotSupported;
  const int nhi = (a.hi_total + a.CHI - 1) / a.CHI;
  const int nlo = (a.lo_total + a.CLO - 1) / a.CLO;
  const long long npanel = (long long)nhi * nlo * a.batch;
  const int sms = sm_count();
  const size_t mo_bytes = a.mul_o ? sizeof(float) * (size_t)a.nout : 0;
  const size_t smem = sizeof(float2) * ((size_t)R::XROWS * CP + (size_t)(a.nin + 1) * CP) + mo_bytes;
  if (npanel < 4LL * sms || npanel >= (1LL << 31) || smem > 220 * 1024 || (long long)nhi * nlo >= (1LL << 22))
    return cudaErrorNotSupported;
  const void* optr = a.out_mag ? static_cast<const void*>(a.out_mag) : static_cast<const void*>(a.out);
  const int in_vec2 = !a.load_i_fastest && a.in_slo == 1 && a.CLO % 2 == 0 && a.lo_total % 2 == 0 &&
                      reinterpret_cast<uintptr_t>(a.in) % 16 == 0 && a.in_sb % 2 == 0 && a.in_si % 2 == 0 &&
                      a.in_shi % 2 == 0;
  const int out_vec2 = a.out_slo == 1 && a.CLO % 2 == 0 && a.lo_total % 2 == 0 &&
                       reinterpret_cast<uintptr_t>(optr) % (a.out_mag ? 8 : 16) == 0 && a.out_sb % 2 == 0 &&
                       a.out_si % 2 == 0 && a.out_shi % 2 == 0;
  auto run = [&](auto kern, int& occ, size_t& occ_smem, bool& configured) -> cudaError_t {
    if (!configured) {
      cudaError_t e = configure(kern, 220 * 1024);
      if (e != cudaSuccess) return e;
      configured = true;
    }
    if (occ_smem != smem) {
      int nb = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, R::NT, smem);
      if (e != cudaSuccess) return e;
      occ = std::max(nb, 1);
      occ_smem = smem;
    }
    const int grid = (int)std::min<long long>(npanel, (long long)sms * occ);
    kern<<<grid, R::NT, smem, s>>>(a, (int)npanel, in_vec2, out_vec2, 0);
    return cudaGetLastError();
  };
  static int occ_f = 1, occ_i = 1;
  static size_t sm_f = 0, sm_i = 0;
  static bool cf = false, ci = false;
  return inverse ? run(panel_fft32_kernel<LOGN, CP, true>, occ_i, sm_i, ci)
                 : run(panel_fft32_kernel<LOGN, CP, false>, occ_f, sm_f, cf);
}

cudaError_t launch_panel_fft_reg(int logn, bool inverse, const PanelArgs& a, cudaStream_t s) {
  switch (logn) {
    case 9: return inverse ? launch_reg<9, 8, true>(a, s) : launch_reg<9, 8, false>(a, s);
    case 10: return inverse ? launch_reg<10, 8, true>(a, s) : launch_reg<10, 8, false>(a, s);
    case 11: return inverse ? launch_reg<11, 4, true>(a, s) : launch_reg<11, 4, false>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_panel_bluestein_reg(int logn, const PanelArgs& a, const float2* cpre, const float2* bhat,
                                       const float2* cpost, cudaStream_t s) {
  switch (logn) {
    case 9: return launch_bluestein_reg<9, 8>(a, cpre, bhat, cpost, s);
    case 10: return launch_bluestein_reg<10, 8>(a, cpre, bhat, cpost, s);
    case 11: return launch_bluestein_reg<11, 4>(a, cpre, bhat, cpost, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nursd
