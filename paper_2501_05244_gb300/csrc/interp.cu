// NUFFT type-2 interpolation (Sec. 6: NUFFT-2 reverses the three type-1 steps,
// the last being interpolation of the blurred signal at the non-uniform points).
//
// After deconvolution and the inverse fine-grid FFT, the value at a point with
// fine coordinate u is sum over its w x w footprint of b[g] phi(2(gx-ux)/w)
// phi(2(gy-uy)/w) -- exactly the adjoint of the spread.
//
// interp_points: relay samples on a channel-last grid [W][W][F]; one warp per
//   sample, one lane per channel, so each tap is a 256-byte coalesced row.  With
//   GRAD the same taps interpolate two more grids, the type-2 grids of kx R and
//   ky R (the spectral derivative), reduced against the sample's phasors into the
//   position gradient.
// interp_planes: voxels of each depth plane on a plane-major grid [Z][W][W];
//   one thread per voxel (rows of w contiguous cells).
#include "nursd_internal.cuh"

namespace nursd {
namespace {

template <int WID, bool GRAD>
__global__ void __launch_bounds__(256) interp_points_kernel(const InterpArgs a) {
  const int slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (slot >= a.L) return;
  const int l = __ldg(a.sorted_l + slot);
  const int2 o = __ldg(a.i0 + slot);
  float wx[WID], wy[WID];
#pragma unroll
  for (int t = 0; t < WID; ++t) {
    wx[t] = __ldg(a.wts + (size_t)slot * 2 * WID + t);
    wy[t] = __ldg(a.wts + (size_t)slot * 2 * WID + WID + t);
  }
  float gsx = 0.f, gsy = 0.f;
  for (int f0 = 0; f0 < a.F; f0 += 32) {
    const int f = f0 + lane;
    if (f >= a.F) break;
    float2 acc = make_float2(0.f, 0.f), ax = make_float2(0.f, 0.f), ay = make_float2(0.f, 0.f);
#pragma unroll
    for (int ty = 0; ty < WID; ++ty) {
      const size_t row = ((size_t)(o.y + ty) * a.W + o.x) * a.F + f;
      float2 rs = make_float2(0.f, 0.f), rx = make_float2(0.f, 0.f), ry = make_float2(0.f, 0.f);
#pragma unroll
      for (int tx = 0; tx < WID; ++tx) {
        const size_t at = row + (size_t)tx * a.F;
        if (a.out) {
          const float2 v = __ldg(a.fine + at);
          rs.x = fmaf(v.x, wx[tx], rs.x);
          rs.y = fmaf(v.y, wx[tx], rs.y);
        }
        if (GRAD) {
          const float2 vx = __ldg(a.fine_dx + at), vy = __ldg(a.fine_dy + at);
          rx.x = fmaf(vx.x, wx[tx], rx.x);
          rx.y = fmaf(vx.y, wx[tx], rx.y);
          ry.x = fmaf(vy.x, wx[tx], ry.x);
          ry.y = fmaf(vy.y, wx[tx], ry.y);
        }
      }
      acc.x = fmaf(rs.x, wy[ty], acc.x);
      acc.y = fmaf(rs.y, wy[ty], acc.y);
      if (GRAD) {
        ax.x = fmaf(rx.x, wy[ty], ax.x);
        ax.y = fmaf(rx.y, wy[ty], ax.y);
        ay.x = fmaf(ry.x, wy[ty], ay.x);
        ay.y = fmaf(ry.y, wy[ty], ay.y);
      }
    }
    if (a.out) a.out[(size_t)l * a.F + f] = make_float2(acc.x * a.scale, acc.y * a.scale);
    if (GRAD) {
      // d/dx of the type-2 value is i (2 pi / (M delta)) times the type 2 of kx R, so
      // Re(p conj(d/dx)) = (2 pi / (M delta)) Im(p conj(ax))
      const float2 p = __ldg(a.P + (size_t)l * a.F + f);
      gsx += p.y * ax.x - p.x * ax.y;
      gsy += p.y * ay.x - p.x * ay.y;
    }
  }
  if (GRAD) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      gsx += __shfl_xor_sync(0xffffffffu, gsx, off);
      gsy += __shfl_xor_sync(0xffffffffu, gsy, off);
    }
    if (lane == 0) {
      const float s = a.scale * a.dudx;
      a.gxy[2 * l] = gsx * s;
      a.gxy[2 * l + 1] = gsy * s;
    }
  }
}

template <int WID>
__global__ void __launch_bounds__(256) interp_planes_kernel(const PlaneInterpArgs a) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)a.Z * a.K) return;
  const int z = (int)(idx / a.K);
  // plane z's lattice pitch is plane_scale[z] times the plan's (the scaled planes of SRSD)
  const double sz = a.plane_scale ? __ldg(a.plane_scale + z) : 1.0;
  const double half = a.half_extent * sz, inv = a.inv_fine_pitch / sz;
  const double dx = (double)a.vox[2 * idx] - a.cx, dy = (double)a.vox[2 * idx + 1] - a.cy;
  if (!(fabs(dx) <= half && fabs(dy) <= half)) {
    atomicOr(a.status, 1);
    a.out[idx] = make_float2(0.f, 0.f);
    return;
  }
  const double ux = dx * inv, uy = dy * inv;
  const int ix = (int)ceil(ux - 0.5 * WID), iy = (int)ceil(uy - 0.5 * WID);
  float wx[WID], wy[WID];
#pragma unroll
  for (int t = 0; t < WID; ++t) {
    const float zx = (float)(((double)(ix + t) - ux) * (2.0 / WID));
    const float zy = (float)(((double)(iy + t) - uy) * (2.0 / WID));
    wx[t] = fabsf(zx) < 1.f ? expf(a.beta * (sqrtf(1.f - zx * zx) - 1.f)) : 0.f;
    wy[t] = fabsf(zy) < 1.f ? expf(a.beta * (sqrtf(1.f - zy * zy) - 1.f)) : 0.f;
  }
  const int rx = min(max(ix - a.g0, 0), a.W - WID), ry = min(max(iy - a.g0, 0), a.W - WID);
  const float2* plane = a.fine + (size_t)z * a.W * a.W;
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int ty = 0; ty < WID; ++ty) {
    const float2* row = plane + (size_t)(ry + ty) * a.W + rx;
    float2 rs = make_float2(0.f, 0.f);
#pragma unroll
    for (int tx = 0; tx < WID; ++tx) {
      const float2 v = __ldg(row + tx);
      rs.x = fmaf(v.x, wx[tx], rs.x);
      rs.y = fmaf(v.y, wx[tx], rs.y);
    }
    acc.x = fmaf(rs.x, wy[ty], acc.x);
    acc.y = fmaf(rs.y, wy[ty], acc.y);
  }
  a.out[idx] = make_float2(acc.x * a.scale, acc.y * a.scale);
}

template <int WID>
cudaError_t points_w(const InterpArgs& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)(((long long)a.L * 32 + 255) / 256);
  if (a.gxy)
    interp_points_kernel<WID, true><<<blocks, 256, 0, s>>>(a);
  else
    interp_points_kernel<WID, false><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <int WID>
cudaError_t planes_w(const PlaneInterpArgs& a, cudaStream_t s) {
  const long long n = (long long)a.Z * a.K;
  interp_planes_kernel<WID><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interp_points(const InterpArgs& a, cudaStream_t s) {
  if (a.L <= 0) return cudaSuccess;
  if (a.gxy && (!a.P || !a.fine_dx || !a.fine_dy)) return cudaErrorInvalidValue;
  switch (a.width) {
    case 4: return points_w<4>(a, s);
    case 5: return points_w<5>(a, s);
    case 6: return points_w<6>(a, s);
    case 7: return points_w<7>(a, s);
    case 8: return points_w<8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_interp_planes(const PlaneInterpArgs& a, cudaStream_t s) {
  if ((long long)a.Z * a.K <= 0) return cudaSuccess;
  switch (a.width) {
    case 4: return planes_w<4>(a, s);
    case 5: return planes_w<5>(a, s);
    case 6: return planes_w<6>(a, s);
    case 7: return planes_w<7>(a, s);
    case 8: return planes_w<8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nursd
