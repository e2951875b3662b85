// RSD transfer-function multiply with the coherent frequency sum (Eq. 4 product,
// frequency integral of Eq. 2): Y_z(k) = sum_f U_f(k) Ghat_{z,f}(k), and its
// adjoint R_f(k) = sum_z conj(Ghat_{z,f}(k)) Y'_z(k).
//
// Generic form: Out[k][j] = sum_r In[k][r] * T[class(k)][r][j] (T conjugated for
// the adjoint), with (r, j) = (f, z) forward on the table Gc[class][f][z] and
// (r, j) = (z, f) for the adjoint on its transposed copy GcT[class][z][f].
//
// Ghat_{z,f} is even in kx and ky and symmetric under kx <-> ky (G depends on
// |j| only), so it is stored once per class {(+-p, +-q), (+-q, +-p)},
// 0 <= q <= p <= M/2, as Gc[class][f][z] -- 1/8 of the full table.  One warp
// owns one class: it stages the class's 8 spectrum rows U[k_s][0..F) in shared
// memory (each a contiguous F-vector), then streams the class's F x Z table
// (contiguous, each lane holding ZPL consecutive depths) once, accumulating
// ZPL x 8 complex sums in registers, and finally writes the 8 depth rows
// Y[k_s][0..Z) (contiguous).  Duplicate members of degenerate classes
// (q = 0, q = p, p = M/2) are recomputed and rewritten with identical values
// by the same lane.  HBM traffic: the table once, U once, Y once.
#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int kClsPerCta = 8;

__device__ __forceinline__ int wrap_index(int k, int M) { return (k + M / 2) & (M - 1); }

// Names follow the forward direction: F is the reduced extent, Z the per-lane one.
// Grid: x = batch item (fastest, so all items of a class group run back to back and
// share the group's table block in L2), y = class group, z = chunk of 32*ZPL outputs.
template <int ZPL, bool CONJ>
__global__ void __launch_bounds__(kClsPerCta * 32, 2) contract_kernel(const float2* __restrict__ U,
                                                                   const float2* __restrict__ Gc,
                                                                   const int2* __restrict__ cls_pq, int ncls, int M,
                                                                   int F, int Z, float2* __restrict__ Y,
                                                                   long long u_stride, long long y_stride) {
  extern __shared__ float4 us4[];  // [kClsPerCta][F][8 slots] complex as float4 pairs
  float2* us = reinterpret_cast<float2*>(us4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.y * kClsPerCta + warp;
  if (c >= ncls) return;
  U += blockIdx.x * u_stride;
  Y += blockIdx.x * y_stride;  // whole warp leaves; nothing below synchronises across warps
  const int2 pq = __ldg(cls_pq + c);
  const int p = pq.x, q = pq.y;
  const int kx[8] = {p, -p, p, -p, q, -q, q, -q};
  const int ky[8] = {q, q, -q, -q, p, p, -p, -p};
  unsigned off[8];  // mode index ky*M + kx of each class member (M <= 1024)
#pragma unroll
  for (int s = 0; s < 8; ++s) off[s] = (unsigned)(wrap_index(ky[s], M) * M + wrap_index(kx[s], M));

  float2* my = us + (size_t)warp * F * 8;
#pragma unroll
  for (int s = 0; s < 8; ++s)
    for (int f = lane; f < F; f += 32) my[f * 8 + s] = __ldg(U + (size_t)off[s] * F + f);
  __syncwarp();

  const int z0 = blockIdx.z * (32 * ZPL) + lane * ZPL;
  float2 acc[ZPL][8];
#pragma unroll
  for (int i = 0; i < ZPL; ++i)
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[i][s] = make_float2(0.f, 0.f);

  const float2* __restrict__ g = Gc + (size_t)c * F * Z + z0;
  // 16-byte vector access needs an even Z (all row offsets are then even)
  const bool full = (z0 + ZPL <= Z) && ((Z & 1) == 0);
  auto load_row = [&](int f, float2* gv) {
    if (f >= F) return;
    if (full && (ZPL % 2 == 0)) {
#pragma unroll
      for (int i = 0; i < ZPL; i += 2) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(g + (size_t)f * Z + i));
        gv[i] = make_float2(t.x, t.y);
        gv[i + 1] = make_float2(t.z, t.w);
      }
    } else {
#pragma unroll
      for (int i = 0; i < ZPL; ++i) gv[i] = (z0 + i < Z) ? __ldg(g + (size_t)f * Z + i) : make_float2(0.f, 0.f);
    }
  };
  // table rows are prefetched kAhead rows ahead of their use, so that each warp keeps
  // about kAhead x 1 KB in flight
  constexpr int kAhead = ZPL == 4 ? 3 : 4;
  float2 ring[kAhead][ZPL];
#pragma unroll
  for (int d = 0; d < kAhead; ++d) load_row(d, ring[d]);
  for (int fb = 0; fb < F; fb += kAhead) {
#pragma unroll
    for (int d = 0; d < kAhead; ++d) {
      const int f = fb + d;
      if (f >= F) break;
      float2 gv[ZPL];
#pragma unroll
      for (int i = 0; i < ZPL; ++i) gv[i] = ring[d][i];
      load_row(f + kAhead, ring[d]);
      if (CONJ) {
#pragma unroll
        for (int i = 0; i < ZPL; ++i) gv[i].y = -gv[i].y;
      }
      const float4* u4 = reinterpret_cast<const float4*>(my + f * 8);
      float2 u[8];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float4 t = u4[s];
        u[2 * s] = make_float2(t.x, t.y);
        u[2 * s + 1] = make_float2(t.z, t.w);
      }
#pragma unroll
      for (int i = 0; i < ZPL; ++i)
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          acc[i][s].x = fmaf(gv[i].x, u[s].x, acc[i][s].x);
          acc[i][s].x = fmaf(-gv[i].y, u[s].y, acc[i][s].x);
          acc[i][s].y = fmaf(gv[i].x, u[s].y, acc[i][s].y);
          acc[i][s].y = fmaf(gv[i].y, u[s].x, acc[i][s].y);
        }
    }
  }
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    float2* dst = Y + (size_t)off[s] * Z + z0;
    if (full && (ZPL % 2 == 0)) {
#pragma unroll
      for (int i = 0; i < ZPL; i += 2)
        *reinterpret_cast<float4*>(dst + i) = make_float4(acc[i][s].x, acc[i][s].y, acc[i + 1][s].x, acc[i + 1][s].y);
    } else {
#pragma unroll
      for (int i = 0; i < ZPL; ++i)
        if (z0 + i < Z) dst[i] = acc[i][s];
    }
  }
}

template <int ZPL, bool CONJ>
cudaError_t launch_zpl(const float2* U, const float2* Gc, const int2* cls_pq, int ncls, int M, int F, int Z,
                       float2* Y, cudaStream_t s, int B = 1, long long u_stride = 0, long long y_stride = 0) {
  const size_t smem = sizeof(float2) * kClsPerCta * F * 8;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(contract_kernel<ZPL, CONJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float2) * kClsPerCta * 256 * 8));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid(B, (ncls + kClsPerCta - 1) / kClsPerCta, (Z + 32 * ZPL - 1) / (32 * ZPL));
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
  contract_kernel<ZPL, CONJ><<<grid, kClsPerCta * 32, smem, s>>>(U, Gc, cls_pq, ncls, M, F, Z, Y, u_stride, y_stride);
  return cudaGetLastError();
}

template <bool CONJ>
cudaError_t launch_dir(const float2* In, const float2* T, const int2* cls_pq, int ncls, int M, int R, int J,
                       float2* Out, cudaStream_t s) {
  if (R > 256) return cudaErrorInvalidValue;
  // outputs per lane (a CTA column covers 32*ZPL of them): 4 for deep extents, fewer for shallow ones.
  if (J > 64) return launch_zpl<4, CONJ>(In, T, cls_pq, ncls, M, R, J, Out, s);
  if (J > 32) return launch_zpl<2, CONJ>(In, T, cls_pq, ncls, M, R, J, Out, s);
  return launch_zpl<1, CONJ>(In, T, cls_pq, ncls, M, R, J, Out, s);
}

}  // namespace

cudaError_t launch_contract(const float2* U, const float2* Gc, const int2* cls_pq, int ncls, int M, int F, int Z,
                            float2* Y, cudaStream_t s) {
  return launch_dir<false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s);
}

cudaError_t launch_contract_batched(const float2* U, long long u_stride, const float2* Gc, const int2* cls_pq,
                                   int ncls, int M, int F, int Z, float2* Y, long long y_stride, int B,
                                   cudaStream_t s) {
  if (F > 256 || B < 1) return cudaErrorInvalidValue;
  if (Z > 64) return launch_zpl<4, false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s, B, u_stride, y_stride);
  if (Z > 32) return launch_zpl<2, false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s, B, u_stride, y_stride);
  return launch_zpl<1, false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s, B, u_stride, y_stride);
}

cudaError_t launch_contract_adjoint(const float2* Yt, const float2* GcT, const int2* cls_pq, int ncls, int M, int F,
                                    int Z, float2* R, cudaStream_t s) {
  return launch_dir<true>(Yt, GcT, cls_pq, ncls, M, Z, F, R, s);
}

}  // namespace nursd
