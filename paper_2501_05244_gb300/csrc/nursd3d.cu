// 3D NURSD for non-planar relays (Eq. 3D_NURSD with Eq. 3d_rsd): the relay samples carry a height h_l
// above or below the reference plane z0, and stage 1 is a 3D type-1 NUFFT of the samples at
// (x_l, y_l, h_l) times the 3D transfer function, evaluated at the plane z0.  The kernels here are
// the pieces that the planar operator does not already have:
//   - the samples' fine coordinate along z (in the spread's slot order) and its range check;
//   - the phasors of one fine z slice: P[l][f] phi(2 (gz - uz_l) / w) (zero off the footprint), so
//     that the planar spread and lateral FFT passes, run once per z slice of the window, give the
//     3D fine grid's lateral spectra slice by slice;
//   - the sum over kz of the 3D spectrum times the 3D transfer function (the slice z = z0 of the
//     inverse transform along z), per lateral mode and frequency.
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

// uz_sorted[s] = fine z coordinate of sorted sample s, h * 2 / dz (the z grid is oversampled by 2);
// |h| > half_extent flags status bit 1 and gives the sample no weight (an origin far outside the window).
__global__ void z_coords_kernel(const float* __restrict__ h_rel, const int* __restrict__ sorted_l, int L,
                                double inv_fine_dz, double half_extent, float* __restrict__ uz_sorted,
                                int* __restrict__ status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= L) return;
  const int l = __ldg(sorted_l + s);
  const double h = (double)__ldg(h_rel + l);
  if (!(fabs(h) <= half_extent)) {
    atomicOr(status, 1);
    uz_sorted[s] = 1e30f;
    return;
  }
  uz_sorted[s] = (float)(h * inv_fine_dz);
}

// Pz[j][s][f] = P[sorted_l[s]][f] phi(2 (gz - uz[s]) / w) for the z cells gz = gz_first + j (blockIdx.y;
// phi the ES kernel, zero for |2 (gz - uz) / w| >= 1), in slot order: one thread per (slot, channel).
__global__ void z_slice_phasors_kernel(const float2* __restrict__ P, const int* __restrict__ sorted_l,
                                       const float* __restrict__ uz, int L, int F, int gz_first, long long pz_stride,
                                       int w, float beta, float2* __restrict__ Pz) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)L * F) return;
  const int gz = gz_first + (int)blockIdx.y;
  Pz += blockIdx.y * pz_stride;
  const int s = (int)(e / F), f = (int)(e % F);
  const float zz = 2.f * ((float)gz - __ldg(uz + s)) / (float)w;
  float2 v = make_float2(0.f, 0.f);
  if (fabsf(zz) < 1.f) {
    const float wt = expf(beta * (sqrtf(1.f - zz * zz) - 1.f));
    const float2 p = __ldg(P + (size_t)__ldg(sorted_l + s) * F + f);
    v = make_float2(p.x * wt, p.y * wt);
  }
  Pz[e] = v;
}

// What[k][f] = scale sum_kz U3[k][kz][f] G3[k][kz][f], k over M^2 lateral modes.
__global__ void kz_sum_kernel(const float2* __restrict__ U3, const float2* __restrict__ G3, long long nk, int Mz,
                              int F, float scale, float2* __restrict__ What) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= nk * F) return;
  const long long k = e / F;
  const int f = (int)(e % F);
  const float2* u = U3 + (size_t)k * Mz * F + f;
  const float2* g = G3 + (size_t)k * Mz * F + f;
  float2 acc = make_float2(0.f, 0.f);
  for (int kz = 0; kz < Mz; ++kz) {
    const float2 a = __ldg(u + (size_t)kz * F), b = __ldg(g + (size_t)kz * F);
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
  }
  What[e] = make_float2(acc.x * scale, acc.y * scale);
}

unsigned blocks_for(long long n) { return (unsigned)std::max<long long>(1, (n + 255) / 256); }

}  // namespace

cudaError_t launch_z_coords(const float* h, const int* sorted_l, int L, double inv_fine_dz, double half_extent,
                            float* uz_sorted, int* status, cudaStream_t s) {
  if (L <= 0) return cudaSuccess;
  z_coords_kernel<<<blocks_for(L), 256, 0, s>>>(h, sorted_l, L, inv_fine_dz, half_extent, uz_sorted, status);
  return cudaGetLastError();
}

cudaError_t launch_z_slice_phasors(const float2* P, const int* sorted_l, const float* uz, int L, int F, int gz_first,
                                   int n, long long pz_stride, int w, float beta, float2* Pz, cudaStream_t s) {
  if (L <= 0) return cudaSuccess;
  if (n < 1 || n > 65535 || pz_stride < (long long)L * F) return cudaErrorInvalidValue;
  z_slice_phasors_kernel<<<dim3(blocks_for((long long)L * F), (unsigned)n), 256, 0, s>>>(P, sorted_l, uz, L, F, gz_first,
                                                                                       pz_stride, w, beta, Pz);
  return cudaGetLastError();
}

cudaError_t launch_kz_sum(const float2* U3, const float2* G3, long long nk, int Mz, int F, float scale, float2* What,
                          cudaStream_t s) {
  kz_sum_kernel<<<blocks_for(nk * F), 256, 0, s>>>(U3, G3, nk, Mz, F, scale, What);
  return cudaGetLastError();
}

}  // namespace nursd
