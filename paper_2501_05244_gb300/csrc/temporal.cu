// Temporal transform to phasors (Eq. PF_Response with the band-pass of Eq. PFPacket).
//
// P[l][f] = w_f sum_n h[l][n] exp(-i w_f (t0 + n dt)) is a real matrix product
// C[L][2F] = H[L][T] * B[T][2F] with B[n][2f] = w_f cos(w_f t_n) and
// B[n][2f+1] = -w_f sin(w_f t_n) (built in FP64 on the host), and C read as
// interleaved complex64 [L][F].  SIMT FP32 tiled GEMM: 128x128 CTA tile, k-step
// 8, double-buffered shared-memory tiles, 8x8 outputs per thread.
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int BM = 128, BN = 128, BK = 8, NT = 256;

struct GemmSmem {
  float As[2][BK][BM + 4];
  float Bs[2][BK][BN];
};

// One 128 x 128 output tile of C = A B (rows m0.., columns n0..).
__device__ __forceinline__ void gemm_tile(GemmSmem& sm, const float* __restrict__ A, const float* __restrict__ B,
                                          float* __restrict__ C, int L, int K, int NC, int m0, int n0) {
  auto& As = sm.As;
  auto& Bs = sm.Bs;
  const int tid = threadIdx.x;
  const int a_row = tid >> 1, a_k = (tid & 1) * 4;     // 128 rows x 8 k as float4
  const int tx = tid & 15, ty = tid >> 4;              // 16 x 16 compute grid

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float4 pa;
  float pb[4];
  auto load_a = [&](int k0) {
    const int r = m0 + a_row;
    pa = (r < L) ? __ldg(reinterpret_cast<const float4*>(A + (size_t)r * K + k0 + a_k)) : make_float4(0, 0, 0, 0);
  };
  auto load_b = [&](int k0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + i * NT;  // 0..1023 over the 8 x 128 tile
      const int kk = e >> 7, c = n0 + (e & 127);
      pb[i] = (c < NC) ? __ldg(B + (size_t)(k0 + kk) * NC + c) : 0.f;
    }
  };
  auto store = [&](int buf) {
    As[buf][a_k + 0][a_row] = pa.x;
    As[buf][a_k + 1][a_row] = pa.y;
    As[buf][a_k + 2][a_row] = pa.z;
    As[buf][a_k + 3][a_row] = pa.w;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + i * NT;
      Bs[buf][e >> 7][e & 127] = pb[i];
    }
  };

  load_a(0);
  load_b(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) {
      load_a(k0 + BK);
      load_b(k0 + BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (r >= L) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (c < NC) C[(size_t)r * NC + c] = acc[i][j];
    }
  }
}

__global__ void __launch_bounds__(NT, 2) sgemm_hb_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                       float* __restrict__ C, int L, int K, int NC) {
  __shared__ __align__(16) GemmSmem sm;
  gemm_tile(sm, A, B, C, L, K, NC, blockIdx.y * BM, blockIdx.x * BN);
}

// Persistent form over a ragged batch: tiles of every item are numbered
// consecutively (item b owns tiles [tile_start[b], tile_start[b+1])), and each
// CTA takes the next tile from a device counter until none are left.
__global__ void __launch_bounds__(NT, 2) sgemm_hb_batched_kernel(const TemporalBatch bt, const float* __restrict__ B,
                                                               int K, int NC, int* __restrict__ counter) {
  __shared__ __align__(16) GemmSmem sm;
  __shared__ int tile;
  const int ncol = (NC + BN - 1) / BN;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) tile = atomicAdd(counter, 1);
    __syncthreads();
    const int t = tile;
    if (t >= bt.tile_start[bt.n]) break;
    int b = 0;
    while (t >= bt.tile_start[b + 1]) ++b;
    const int local = t - bt.tile_start[b];
    gemm_tile(sm, bt.A[b], B, bt.C[b], bt.L[b], K, NC, (local / ncol) * BM, (local % ncol) * BN);
  }
}

}  // namespace

cudaError_t launch_temporal_dft_batched(const TemporalBatch& bt, const float* B, int T, int twoF, int* counter,
                                        cudaStream_t s) {
  if (T % BK != 0 || bt.n < 1 || bt.n > kMaxBatch) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = bt.tile_start[bt.n];
  const int grid = std::max(1, std::min(tiles, 2 * sms));
  sgemm_hb_batched_kernel<<<grid, NT, 0, s>>>(bt, B, T, twoF, counter);
  return cudaGetLastError();
}

cudaError_t launch_temporal_dft(const float* h, const float* B, float* C, int L, int T, int twoF, cudaStream_t s) {
  if (L <= 0) return cudaSuccess;
  if (T % BK != 0) return cudaErrorInvalidValue;
  dim3 grid((twoF + BN - 1) / BN, (L + BM - 1) / BM);
  sgemm_hb_kernel<<<grid, NT, 0, s>>>(h, B, C, L, T, twoF);
  return cudaGetLastError();
}

}  // namespace nursd
