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
                                    const double* __restrict__ k, int F, long long total) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int f = (int)(idx % F);
  long long rest = idx / F;
  const int zb = (int)(rest % ZB);
  rest /= ZB;
  const int jx = (int)(rest % M), jy = (int)(rest / M);
  const double x = (double)(jx - M / 2) * pitch, y = (double)(jy - M / 2) * pitch, zz = z[zb];
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

}  // namespace

cudaError_t launch_gtf_generate(float2* g, int M, double pitch, const double* d_z, int ZB, const double* d_k, int F,
                                cudaStream_t s) {
  const long long total = (long long)M * M * ZB * F;
  gtf_generate_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, M, pitch, d_z, ZB, d_k, F, total);
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
