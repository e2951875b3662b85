// Per-frequency forms of the operator: the single-illumination volume (Eq. PF_RSD_Defn with the
// illumination phase mask of one illumination point x_p) and time-resolved frames of the virtual
// wave (Eq. Video_Voxel_Freq_Offset).  Both weight each frequency's reconstruction
//   V_{z,f}[m] = M^-2 sum_k U_f(k) Ghat_{z,f}(k) exp(+2 pi i k.m / M),  m in I_N^2,
// by a factor that varies with the voxel (exp(+i k_f |x_p - x_v|)) or with the frame
// (exp(+i w_f t)), so the frequency sum cannot be taken before the inverse transform as in the
// ordinary path.  For a group of zg depths at a time the plan forms the products U_f Ghat_{z,f}
// (transfer_depths_kernel, no sum over f), runs the ordinary path's two pruned inverse passes
// over all zg*F channels into a channel-major buffer [zg F][N][N], and reduces over f with the
// weights (illum_sum_kernel, frames_sum_kernel).
#include "nursd_internal.cuh"

namespace nursd {
namespace {

// Symmetry class of mode (kx, ky): {(+-p, +-q), (+-q, +-p)}, 0 <= q <= p, index p(p+1)/2 + q.
__device__ __forceinline__ int class_of(int kx, int ky) {
  const int a = abs(kx), b = abs(ky);
  const int p = max(a, b), q = min(a, b);
  return p * (p + 1) / 2 + q;
}

// Y[k][zz F + f] = U[k][f] * Gc[class(k)][f][z0 + zz] for zz < zg, with mode k stored at
// (ky + M/2) M + (kx + M/2).  One thread per (k, f): the U read and the Y writes are coalesced
// over f; the zg table values of (class, f) are contiguous.
__global__ void transfer_depths_kernel(const float2* __restrict__ U, const float2* __restrict__ Gc, int M, int F,
                                       int Z, int z0, int zg, float2* __restrict__ Y) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)M * M * F) return;
  const int f = (int)(idx % F);
  const long long k = idx / F;
  const int kx = (int)(k % M) - M / 2, ky = (int)(k / M) - M / 2;
  const float2 u = __ldg(U + idx);
  const float2* g = Gc + ((size_t)class_of(kx, ky) * F + f) * Z + z0;
  float2* y = Y + k * (long long)zg * F + f;
  for (int zz = 0; zz < zg; ++zz) {
    const float2 t = __ldg(g + zz);
    y[(size_t)zz * F] = make_float2(u.x * t.x - u.y * t.y, u.x * t.y + u.y * t.x);
  }
}

// exp(+2 pi i t) for t in cycles, reduced to [-1/2, 1/2] in FP64 before the FP32 sincospi.
__device__ __forceinline__ float2 phasor_cycles(double t) {
  const float r = (float)(t - rint(t));
  float sn, cs;
  sincospif(2.f * r, &sn, &cs);
  return make_float2(cs, sn);
}

constexpr int kReseed = 16;  // recurrence steps between FP64 re-evaluations of the mask

// out[z0 + zz][my][mx] = sum_f exp(+i k_f |x_p - x_v|) V[zz cz + f cf][my][mx], one thread per voxel,
// x_v = (cx + (mx - N/2) pitch, cy + (my - N/2) pitch, depth[z0 + zz]).  k_f = 2 pi kap[f]; the
// distance and each phase in cycles are taken in FP64 (|k d| reaches hundreds of radians).  With
// equispaced frequencies (kap[f] = kap0 + f dkap) the mask advances by one complex rotation per
// frequency and is re-evaluated in FP64 every kReseed frequencies; otherwise every phase is.
__global__ void illum_sum_kernel(const float2* __restrict__ V, int F, int N, int z0, int zg, int cz, int cf,
                                 IllumArgs a, float2* __restrict__ out) {
  const int nn = N * N;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= zg * nn) return;
  const int zz = idx / nn, m = idx - zz * nn;
  const int my = m / N, mx = m - my * N;
  const double dx = a.cx + (double)(mx - N / 2) * a.pitch - a.xp;
  const double dy = a.cy + (double)(my - N / 2) * a.pitch - a.yp;
  const double dz = __ldg(a.depth + z0 + zz) - a.zp;
  const double d = sqrt(dx * dx + dy * dy + dz * dz);
  const float2* v = V + (size_t)zz * cz * nn + m;
  const size_t fs = (size_t)cf * nn;  // from one frequency's channel to the next
  float2 acc = make_float2(0.f, 0.f);
  if (a.equispaced) {
    const float2 rot = phasor_cycles(a.dkap * d);
    for (int f0 = 0; f0 < F; f0 += kReseed) {
      float2 ph = phasor_cycles(__ldg(a.kap + f0) * d);
      const int f1 = min(F, f0 + kReseed);
      for (int f = f0; f < f1; ++f) {
        const float2 x = __ldg(v + f * fs);
        acc.x = fmaf(ph.x, x.x, fmaf(-ph.y, x.y, acc.x));
        acc.y = fmaf(ph.x, x.y, fmaf(ph.y, x.x, acc.y));
        ph = cmul(ph, rot);
      }
    }
  } else {
    for (int f = 0; f < F; ++f) {
      const float2 ph = phasor_cycles(__ldg(a.kap + f) * d);
      const float2 x = __ldg(v + f * fs);
      acc.x = fmaf(ph.x, x.x, fmaf(-ph.y, x.y, acc.x));
      acc.y = fmaf(ph.x, x.y, fmaf(ph.y, x.x, acc.y));
    }
  }
  out[(size_t)(z0 + zz) * nn + m] = acc;
}

// The same sum with V channel-last [N][N][zg F] and the channel of depth zz and frequency f at
// f zg + zz: one thread per (voxel, depth), depth fastest, so the zg threads of a voxel read its zg
// channels of one frequency as one contiguous run (a 32-byte sector at zg = 4) and the next
// frequency's run follows in the same cache line.  The mask as in illum_sum_kernel.
__global__ void illum_sum_cl_kernel(const float2* __restrict__ V, int F, int N, int z0, int zg, IllumArgs a,
                                    float2* __restrict__ out) {
  const int nn = N * N;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)zg * nn) return;
  const int m = (int)(idx / zg), zz = (int)(idx - (long long)m * zg);
  const int my = m / N, mx = m - my * N;
  const double dx = a.cx + (double)(mx - N / 2) * a.pitch - a.xp;
  const double dy = a.cy + (double)(my - N / 2) * a.pitch - a.yp;
  const double dz = __ldg(a.depth + z0 + zz) - a.zp;
  const double d = sqrt(dx * dx + dy * dy + dz * dz);
  const float2* v = V + (size_t)m * zg * F + zz;
  float2 acc = make_float2(0.f, 0.f);
  if (a.equispaced) {
    const float2 rot = phasor_cycles(a.dkap * d);
    for (int f0 = 0; f0 < F; f0 += kReseed) {
      float2 ph = phasor_cycles(__ldg(a.kap + f0) * d);
      const int f1 = min(F, f0 + kReseed);
#pragma unroll 4
      for (int f = f0; f < f1; ++f) {
        const float2 x = __ldg(v + (size_t)f * zg);
        acc.x = fmaf(ph.x, x.x, fmaf(-ph.y, x.y, acc.x));
        acc.y = fmaf(ph.x, x.y, fmaf(ph.y, x.x, acc.y));
        ph = cmul(ph, rot);
      }
    }
  } else {
    for (int f = 0; f < F; ++f) {
      const float2 ph = phasor_cycles(__ldg(a.kap + f) * d);
      const float2 x = __ldg(v + (size_t)f * zg);
      acc.x = fmaf(ph.x, x.x, fmaf(-ph.y, x.y, acc.x));
      acc.y = fmaf(ph.x, x.y, fmaf(ph.y, x.x, acc.y));
    }
  }
  out[(size_t)(z0 + zz) * nn + m] = acc;
}

constexpr int kFrameChunk = 8;  // frames accumulated per pass over a voxel's F values

// out[t][z0 + zz][my][mx] = sum_f A[t][f] V[zz cz + f cf][my][mx] for t < T, A[t][f] = exp(+i w_f t_t)
// (evaluated in FP64 on the host).  One thread per voxel, kFrameChunk frames per pass.
__global__ void frames_sum_kernel(const float2* __restrict__ V, int F, int N, int Z, int z0, int zg, int cz, int cf,
                                  const float2* __restrict__ A, int T, float2* __restrict__ out) {
  const int nn = N * N;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= zg * nn) return;
  const int zz = idx / nn, m = idx - zz * nn;
  const float2* v = V + (size_t)zz * cz * nn + m;
  const size_t fs = (size_t)cf * nn;
  for (int t0 = 0; t0 < T; t0 += kFrameChunk) {
    float2 acc[kFrameChunk];
#pragma unroll
    for (int j = 0; j < kFrameChunk; ++j) acc[j] = make_float2(0.f, 0.f);
    const int nt = min(kFrameChunk, T - t0);
    for (int f = 0; f < F; ++f) {
      const float2 x = __ldg(v + f * fs);
#pragma unroll
      for (int j = 0; j < kFrameChunk; ++j) {
        if (j < nt) {
          const float2 w = __ldg(A + (size_t)(t0 + j) * F + f);
          acc[j].x = fmaf(w.x, x.x, fmaf(-w.y, x.y, acc[j].x));
          acc[j].y = fmaf(w.x, x.y, fmaf(w.y, x.x, acc[j].y));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kFrameChunk; ++j)
      if (j < nt) out[((size_t)(t0 + j) * Z + z0 + zz) * nn + m] = acc[j];
  }
}

}  // namespace

cudaError_t launch_transfer_depths(const float2* U, const float2* Gc, int M, int F, int Z, int z0, int zg, float2* Y,
                                   cudaStream_t s) {
  if (M < 2 || F < 1 || zg < 1 || z0 < 0 || z0 + zg > Z) return cudaErrorInvalidValue;
  const long long n = (long long)M * M * F;
  const int threads = 256;
  const long long blocks = (n + threads - 1) / threads;
  if (blocks >= (1LL << 31)) return cudaErrorInvalidValue;
  transfer_depths_kernel<<<(unsigned)blocks, threads, 0, s>>>(U, Gc, M, F, Z, z0, zg, Y);
  return cudaGetLastError();
}

cudaError_t launch_illum_sum(const float2* V, int F, int N, int z0, int zg, int cz, int cf, const IllumArgs& a,
                             float2* out, cudaStream_t s) {
  const long long n = (long long)zg * N * N;
  if (F < 1 || N < 1 || zg < 1 || n >= (1LL << 31)) return cudaErrorInvalidValue;
  const int threads = 256;
  illum_sum_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(V, F, N, z0, zg, cz, cf, a, out);
  return cudaGetLastError();
}

cudaError_t launch_illum_sum_cl(const float2* V, int F, int N, int z0, int zg, const IllumArgs& a, float2* out,
                                cudaStream_t s) {
  const long long threads = (long long)N * N * zg;
  if (F < 1 || N < 1 || zg < 1 || threads >= (1LL << 31)) return cudaErrorInvalidValue;
  illum_sum_cl_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(V, F, N, z0, zg, a, out);
  return cudaGetLastError();
}

cudaError_t launch_frames_sum(const float2* V, int F, int N, int Z, int z0, int zg, int cz, int cf, const float2* A,
                              int T, float2* out, cudaStream_t s) {
  const long long n = (long long)zg * N * N;
  if (F < 1 || N < 1 || zg < 1 || T < 1 || n >= (1LL << 31)) return cudaErrorInvalidValue;
  const int threads = 256;
  frames_sum_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(V, F, N, Z, z0, zg, cz, cf, A, T,
                                                                                out);
  return cudaGetLastError();
}

}  // namespace nursd
