// Transfer-function table (plan time): Ghat_{z,f} = DFT_M[ G(j delta, z, w_f) ],
// G = exp(+i k r) / r, r = sqrt(|j delta|^2 + z^2), j in I_M^2 (Eq. RSD_conv, Eq. 4).
//
// The phase k_f r reaches several hundred radians, so it is formed and reduced
// modulo 2 pi in FP64 before an FP32 sincos; the 2-D DFT then runs through the
// panel FFT in FP32, and the result is compressed to one value per class of
// the 8-fold symmetry (kx, ky) -> (+-kx, +-ky), (ky, kx).
#include "nursd_internal.cuh"

namespace nursd {
namespace {

__global__ void gtf_generate_kernel(float2* __restrict__ g, int M, double pitch, const double* __restrict__ z, int ZB,
                                    const double* __restrict__ k, int F, long long total,
                                    const double* __restrict__ zpitch) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int f = (int)(idx % F);
  long long rest = idx / F;
  const int zb = (int)(rest % ZB);
  rest /= ZB;
  const int jx = (int)(rest % M), jy = (int)(rest / M);
  const double d = zpitch ? zpitch[zb] : pitch;
  const double x = (double)(jx - M / 2) * d, y = (double)(jy - M / 2) * d, zz = z[zb];
  const double r = sqrt(x * x + y * y + zz * zz);
  const double two_pi = 6.283185307179586476925286766559;
  double ph = k[f] * r;
  ph -= two_pi * rint(ph * (1.0 / two_pi));
  float sn, cs;
  sincosf((float)ph, &sn, &cs);
  const float a = (float)(1.0 / r);
  g[idx] = make_float2(a * cs, a * sn);
}

__global__ void gtf_compress_kernel(const float2* __restrict__ Gfull, const int2* __restrict__ cls_pq, int ncls,
                                    int M, int F, int ZB, int Z, int z0, float2* __restrict__ Gc,
                                    float2* __restrict__ GcT) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)ncls * F * ZB;
  if (idx >= total) return;
  const int zb = (int)(idx % ZB);
  const int f = (int)((idx / ZB) % F);
  const int c = (int)(idx / ((long long)ZB * F));
  const int2 pq = cls_pq[c];
  const int ix = (pq.x + M / 2) & (M - 1), iy = (pq.y + M / 2) & (M - 1);  // representative (kx, ky) = (p, q)
  const float2 v = Gfull[((size_t)iy * M + ix) * ZB * F + (size_t)zb * F + f];
  Gc[((size_t)c * F + f) * Z + z0 + zb] = v;
  if (GcT) GcT[((size_t)c * Z + z0 + zb) * F + f] = v;
}

__global__ void gtf_compress_depthmajor_kernel(const float2* __restrict__ Gfull, const int2* __restrict__ cls_pq,
                                               int ncls, int M, int F, int ZB, int z0, float2* __restrict__ Gs) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)ncls * F * ZB;
  if (idx >= total) return;
  const int f = (int)(idx % F);
  const int c = (int)((idx / F) % ncls);
  const int zb = (int)(idx / ((long long)F * ncls));
  const int2 pq = cls_pq[c];
  const int ix = (pq.x + M / 2) & (M - 1), iy = (pq.y + M / 2) & (M - 1);
  Gs[((size_t)(z0 + zb) * ncls + c) * F + f] = Gfull[((size_t)iy * M + ix) * ZB * F + (size_t)zb * F + f];
}

// One warp per class, lanes over frequencies, a shuffle reduction per class member.
__global__ void __launch_bounds__(256) contract_depth_kernel(const float2* __restrict__ Phat,
                                                             const float2* __restrict__ Gs_z,
                                                             const int2* __restrict__ cls_pq, int ncls, int M, int F,
                                                             int Z, int z, float2* __restrict__ Y) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= ncls) return;
  const int2 pq = __ldg(cls_pq + c);
  const int p = pq.x, q = pq.y;
  const int kx[8] = {p, -p, p, -p, q, -q, q, -q};
  const int ky[8] = {q, q, -q, -q, p, p, -p, -p};
  float2 acc[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) acc[s] = make_float2(0.f, 0.f);
  unsigned off[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) off[s] = (unsigned)((((ky[s] + M / 2) & (M - 1)) * M) + ((kx[s] + M / 2) & (M - 1)));
  for (int f = lane; f < F; f += 32) {
    const float2 g = __ldg(Gs_z + (size_t)c * F + f);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const float2 u = __ldg(Phat + (size_t)off[s] * F + f);
      acc[s].x = fmaf(u.x, g.x, fmaf(-u.y, g.y, acc[s].x));
      acc[s].y = fmaf(u.x, g.y, fmaf(u.y, g.x, acc[s].y));
    }
  }
#pragma unroll
  for (int s = 0; s < 8; ++s)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[s].x += __shfl_xor_sync(0xffffffffu, acc[s].x, o);
      acc[s].y += __shfl_xor_sync(0xffffffffu, acc[s].y, o);
    }
  if (lane < 8) {
    float2 v = acc[0];
#pragma unroll
    for (int s = 1; s < 8; ++s)
      if (lane == s) v = acc[s];
    Y[(size_t)off[lane] * Z + z] = v;
  }
}

}  // namespace

cudaError_t launch_gtf_generate(float2* g, int M, double pitch, const double* d_z, int ZB, const double* d_k, int F,
                                cudaStream_t s, const double* d_pitch) {
  const long long total = (long long)M * M * ZB * F;
  gtf_generate_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, M, pitch, d_z, ZB, d_k, F, total, d_pitch);
  return cudaGetLastError();
}

cudaError_t launch_gtf_compress_depthmajor(const float2* Gfull, const int2* cls_pq, int ncls, int M, int F, int ZB,
                                           int z0, float2* Gs, cudaStream_t s) {
  const long long total = (long long)ncls * F * ZB;
  gtf_compress_depthmajor_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Gfull, cls_pq, ncls, M, F, ZB, z0,
                                                                                  Gs);
  return cudaGetLastError();
}

cudaError_t launch_contract_depth(const float2* Phat, const float2* Gs_z, const int2* cls_pq, int ncls, int M, int F,
                                  int Z, int z, float2* Y, cudaStream_t s) {
  const long long threads = (long long)ncls * 32;
  contract_depth_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(Phat, Gs_z, cls_pq, ncls, M, F, Z, z, Y);
  return cudaGetLastError();
}

cudaError_t launch_gtf_compress(const float2* Gfull, const int2* cls_pq, int ncls, int M, int F, int ZB, int Z,
                                int z0, float2* Gc, float2* GcT, cudaStream_t s) {
  const long long total = (long long)ncls * F * ZB;
  gtf_compress_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(Gfull, cls_pq, ncls, M, F, ZB, Z, z0, Gc,
                                                                       GcT);
  return cudaGetLastError();
}

}  // namespace nursd
