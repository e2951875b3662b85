// Temporal transform on the tensor cores (Eq. PF_Response with Eq. PFPacket):
// C[L][2F] = H[L][T] * B[T][2F] * diag(w), B[n][2f] = cos(w_f t_n), B[n][2f+1] = -sin(w_f t_n);
// the weight w_f of each column pair is applied to the accumulator as it is stored.
//
// FP32 accuracy from FP16 tensor-core products: every operand is split into an
// fp16 head and tail, x = x_hi + x_lo with x_lo = fp16(x - x_hi), so x_hi + x_lo
// carries ~22 significant bits, and
//   C = H_hi B_hi + H_hi B_lo + H_lo B_hi
// with every product exact in the FP32 accumulator (11-bit x 11-bit mantissas).
// The twiddle matrix is split once at plan time (stored transposed, [2F][T]);
// histogram tiles are split as they are staged.  Photon counts below 2048 are
// exact in fp16, so a CTA-wide vote drops the H_lo product for such tiles.
//
// FP32 range: the head and tail carry ~22 bits of each value of a row whose max |h| lies in
// [2^-3, 65504).  Each row's max is reduced as the tile is staged; a row outside that window is
// listed (row, exponent e, batch item), and a gather launch recomputes the listed rows from
// h 2^-e (an exact scaling into [2^14, 2^15)) and multiplies the result by 2^e.
//
// mma.sync m16n8k16 (row.col, f16 x f16 -> f32): CTA tile 128 x 128, k-step 32,
// 8 warps of 32 x 64 each, fragments loaded with ldmatrix from padded shared
// memory, the next k-step's tiles staged while the current one is multiplied.
#include <cuda_fp16.h>

#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int BM = 128, BN = 128, BK = 32, NT = 256;
constexpr int LDS = BK + 8;  // padded row (halves): 80 bytes, rows 16-byte aligned

struct TcSmem {
  __half a_hi[BM][LDS];
  __half a_lo[BM][LDS];
  __half b_hi[BN][LDS];
  __half b_lo[BN][LDS];
  // the tile's rows: histogram row (null: zeros), output row (null: not stored), the gather
  // launch's scale exponent, and the (row, item) a detected row is listed under
  const float* src[BM];
  float* dst[BM];
  int rexp[BM];
  int rid[BM];
  int item;
  int any_lo;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma16816(float* c, const unsigned* a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Registers holding one k-step's global data before it is split and stored.
struct Stage {
  float4 a[4];   // 128 x 32 fp32 of H: 16 floats per thread
  uint4 bh[2];   // 128 x 32 fp16 of B_hi^T: 2 x 8 halves per thread
  uint4 bl[2];
};

__device__ __forceinline__ void load_stage(Stage& st, const TcSmem& sm, const __half* __restrict__ Bh,
                                           const __half* __restrict__ Bl, int K, int NC, int n0, int k0) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 4; ++i) {  // A: 128 rows x 8 float4
    const int e = tid + i * NT, r = e >> 3, c4 = (e & 7) * 4;
    const int col = k0 + c4;
    const float* src = sm.src[r];
    st.a[i] = (src && col < K) ? __ldg(reinterpret_cast<const float4*>(src + col)) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {  // B^T: 128 rows (n) x 4 uint4 (8 halves each)
    const int e = tid + i * NT, r = e >> 2, c8 = (e & 3) * 8;
    const int n = n0 + r, col = k0 + c8;
    const bool ok = n < NC && col < K;
    st.bh[i] = ok ? __ldg(reinterpret_cast<const uint4*>(Bh + (size_t)n * K + col)) : make_uint4(0, 0, 0, 0);
    st.bl[i] = ok ? __ldg(reinterpret_cast<const uint4*>(Bl + (size_t)n * K + col)) : make_uint4(0, 0, 0, 0);
  }
}

// Splits and stores one k-step; GATHER scales row r by 2^-rexp[r] first, otherwise the
// running max |h| of this thread's four rows is updated.
template <bool GATHER>
__device__ __forceinline__ void store_stage(TcSmem& sm, const Stage& st, float (&rmax)[4]) {
  const int tid = threadIdx.x;
  int lo_nonzero = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + i * NT, r = e >> 3, c4 = (e & 7) * 4;
    float v[4] = {st.a[i].x, st.a[i].y, st.a[i].z, st.a[i].w};
    if (GATHER) {
      const int x = sm.rexp[r];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = ldexpf(v[j], -x);
    } else {
      rmax[i] = fmaxf(rmax[i], fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3]))));
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __half h = __float2half_rn(v[j]);
      const __half l = __float2half_rn(v[j] - __half2float(h));
      sm.a_hi[r][c4 + j] = h;
      sm.a_lo[r][c4 + j] = l;
      lo_nonzero |= (__half_as_ushort(l) & 0x7fff) != 0;
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int e = tid + i * NT, r = e >> 2, c8 = (e & 3) * 8;
    *reinterpret_cast<uint4*>(&sm.b_hi[r][c8]) = st.bh[i];
    *reinterpret_cast<uint4*>(&sm.b_lo[r][c8]) = st.bl[i];
  }
  if (lo_nonzero) sm.any_lo = 1;
}

// One 128 x 128 output tile of the rows described in sm (filled and synchronised by the caller).
// detect: list the rows whose max |h| lies outside the split's window (done by column tile 0).
template <bool GATHER>
__device__ __forceinline__ void tc_tile(TcSmem& sm, const __half* __restrict__ Bh, const __half* __restrict__ Bl,
                                        const float* __restrict__ wcol, int K, int NC, int n0, bool detect,
                                        const TemporalFix& fix) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = (warp & 3) * 32, wn = (warp >> 2) * 64;  // warp tile origin (4 x 2 warps)
  float acc[2][8][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  float rmax[4] = {0.f, 0.f, 0.f, 0.f};

  Stage st;
  load_stage(st, sm, Bh, Bl, K, NC, n0, 0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    __syncthreads();  // previous k-step's fragments are consumed
    if (tid == 0) sm.any_lo = 0;
    __syncthreads();
    store_stage<GATHER>(sm, st, rmax);
    if (k0 + BK < K) load_stage(st, sm, Bh, Bl, K, NC, n0, k0 + BK);  // overlaps the MMAs below
    __syncthreads();
    const bool use_lo = sm.any_lo != 0;
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned ah[2][4], al[2][4];
      const int ar = lane & 15, ac = kk + (lane >> 4) * 8;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        ldsm_x4(ah[i][0], ah[i][1], ah[i][2], ah[i][3], &sm.a_hi[wm + i * 16 + ar][ac]);
        if (use_lo) ldsm_x4(al[i][0], al[i][1], al[i][2], al[i][3], &sm.a_lo[wm + i * 16 + ar][ac]);
      }
      // B fragments: x4 covers two n8 tiles x k16 (matrices: n0-7 k0-7, n0-7 k8-15, n8-15 k0-7, n8-15 k8-15)
      const int br = (lane & 7) + ((lane >> 4) << 3), bc = kk + ((lane >> 3) & 1) * 8;
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        unsigned h0, h1, h2, h3, l0, l1, l2, l3;
        ldsm_x4(h0, h1, h2, h3, &sm.b_hi[wn + j * 8 + br][bc]);
        ldsm_x4(l0, l1, l2, l3, &sm.b_lo[wn + j * 8 + br][bc]);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          mma16816(acc[i][j], ah[i], h0, h1);
          mma16816(acc[i][j], ah[i], l0, l1);
          mma16816(acc[i][j + 1], ah[i], h2, h3);
          mma16816(acc[i][j + 1], ah[i], l2, l3);
          if (use_lo) {
            mma16816(acc[i][j], al[i], h0, h1);
            mma16816(acc[i][j + 1], al[i], h2, h3);
          }
        }
      }
    }
  }
  if (!GATHER && detect) {  // the 8 lanes tid & ~7 .. tid | 7 share each of the four rows
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float m = rmax[i];
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
      const int r = (tid + i * NT) >> 3;
      if ((tid & 7) == 0 && sm.src[r]) {
        const int x = temporal_row_exponent(m);
        if (x != kRowInRange) {
          const int slot = atomicAdd(fix.count, 1);
          if (slot < fix.cap) fix.list[slot] = make_int4(sm.rid[r], x, sm.item, 0);
        }
      }
    }
  }
  // C fragment: rows g, g+8 (g = lane/4), columns 2 (lane%4) + {0,1}
  const int g = lane >> 2, c2 = (lane & 3) * 2;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = n0 + wn + j * 8 + c2;
      const float w0 = col < NC ? __ldg(wcol + col) : 0.f;
      const float w1 = col + 1 < NC ? __ldg(wcol + col + 1) : 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = wm + i * 16 + g + h * 8;
        float* dst = sm.dst[r];
        if (!dst) continue;
        float v0 = acc[i][j][2 * h] * w0, v1 = acc[i][j][2 * h + 1] * w1;
        if (GATHER) {
          v0 = ldexpf(v0, sm.rexp[r]);
          v1 = ldexpf(v1, sm.rexp[r]);
        }
        if (col + 1 < NC) {
          *reinterpret_cast<float2*>(dst + col) = make_float2(v0, v1);
        } else if (col < NC) {
          dst[col] = v0;
        }
      }
    }
}

// Rows of one tile of item b: H rows m0 .. m0 + 127 of A (L rows), output rows of C (through
// row_slot when given).
__device__ __forceinline__ void rows_direct(TcSmem& sm, const float* A, float* C, int L, int K, int NC, int m0,
                                            int b, const int* __restrict__ row_slot) {
  if (threadIdx.x < BM) {
    const int r = threadIdx.x, row = m0 + r;
    const bool ok = row < L;
    sm.src[r] = ok ? A + (size_t)row * K : nullptr;
    sm.dst[r] = ok ? C + (size_t)(row_slot ? __ldg(row_slot + row) : row) * NC : nullptr;
    sm.rexp[r] = 0;
    sm.rid[r] = row;
  }
  if (threadIdx.x == 0) sm.item = b;
}

__global__ void __launch_bounds__(NT) temporal_tc_kernel(const float* __restrict__ A, const __half* __restrict__ Bh,
                                                        const __half* __restrict__ Bl, const float* __restrict__ wcol,
                                                        float* __restrict__ C, int L, int K, int NC,
                                                        const int* __restrict__ row_slot, const TemporalFix fix) {
  extern __shared__ __align__(16) unsigned char raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(raw);
  rows_direct(sm, A, C, L, K, NC, blockIdx.y * BM, 0, row_slot);
  __syncthreads();
  tc_tile<false>(sm, Bh, Bl, wcol, K, NC, blockIdx.x * BN, blockIdx.x == 0, fix);
}

// Persistent form over a ragged batch (tiles numbered consecutively across items,
// taken from a device counter).
__global__ void __launch_bounds__(NT) temporal_tc_batched_kernel(const TemporalBatch bt, const __half* __restrict__ Bh,
                                                                const __half* __restrict__ Bl,
                                                                const float* __restrict__ wcol, int K, int NC,
                                                                int* __restrict__ counter, const TemporalFix fix) {
  extern __shared__ __align__(16) unsigned char raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(raw);
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
    rows_direct(sm, bt.A[b], bt.C[b], bt.L[b], K, NC, (local / ncol) * BM, b, nullptr);
    __syncthreads();
    tc_tile<false>(sm, Bh, Bl, wcol, K, NC, (local % ncol) * BN, local % ncol == 0, fix);
  }
}

// Gather launch: recomputes the rows listed by the first launch (item, row, exponent), each scaled
// by 2^-e; tiles of 128 listed rows x 128 columns, grid-strided.  row_slot applies to item 0.
__global__ void __launch_bounds__(NT) temporal_tc_gather_kernel(const TemporalBatch bt, const __half* __restrict__ Bh,
                                                               const __half* __restrict__ Bl,
                                                               const float* __restrict__ wcol, int K, int NC,
                                                               const int* __restrict__ row_slot,
                                                               const TemporalFix fix) {
  extern __shared__ __align__(16) unsigned char raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(raw);
  __shared__ int listed;
  if (threadIdx.x == 0) listed = temporal_fix_take(fix);
  __syncthreads();
  const int n = min(listed, fix.cap);
  const int ncol = (NC + BN - 1) / BN, ntiles = (n + BM - 1) / BM * ncol;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();  // the previous tile's epilogue is done with the row table
    if (threadIdx.x < BM) {
      const int r = threadIdx.x, pos = (t / ncol) * BM + r;
      const float* src = nullptr;
      float* dst = nullptr;
      int x = 0;
      if (pos < n) {
        const int4 en = fix.list[pos];
        if (en.z >= 0 && en.z < bt.n && en.x >= 0 && en.x < bt.L[en.z]) {
          src = bt.A[en.z] + (size_t)en.x * K;
          const int orow = (row_slot && en.z == 0) ? __ldg(row_slot + en.x) : en.x;
          dst = bt.C[en.z] + (size_t)orow * NC;
          x = en.y;
        }
      }
      sm.src[r] = src;
      sm.dst[r] = dst;
      sm.rexp[r] = x;
      sm.rid[r] = pos;
    }
    if (threadIdx.x == 0) sm.item = 0;
    __syncthreads();
    tc_tile<true>(sm, Bh, Bl, wcol, K, NC, (t % ncol) * BN, false, fix);
  }
}

bool g_configured = false;
cudaError_t configure() {
  if (g_configured) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(temporal_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(TcSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(temporal_tc_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TcSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(temporal_tc_gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(TcSmem));
  if (e == cudaSuccess) g_configured = true;
  return e;
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

cudaError_t launch_gather(const TemporalBatch& bt, const void* Bh, const void* Bl, const float* wcol, int T, int twoF,
                          int max_rows, const TemporalFix& fix, const int* row_slot, cudaStream_t s) {
  const int rows = std::min(max_rows, fix.cap);
  if (rows <= 0) return cudaSuccess;
  const int ncol = (twoF + BN - 1) / BN;
  const int grid = std::max(1, std::min((rows + BM - 1) / BM * ncol, 2 * sm_count()));
  temporal_tc_gather_kernel<<<grid, NT, sizeof(TcSmem), s>>>(bt, static_cast<const __half*>(Bh),
                                                              static_cast<const __half*>(Bl), wcol, T, twoF, row_slot,
                                                              fix);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_temporal_tc(const float* h, const void* Bh, const void* Bl, const float* wcol, float* C, int L,
                               int T, int twoF, const TemporalFix& fix, cudaStream_t s, const int* row_slot) {
  if (L <= 0) return cudaSuccess;
  if (T % 8 != 0) return cudaErrorInvalidValue;
  cudaError_t e = configure();
  if (e != cudaSuccess) return e;
  dim3 grid((twoF + BN - 1) / BN, (L + BM - 1) / BM);
  temporal_tc_kernel<<<grid, NT, sizeof(TcSmem), s>>>(h, static_cast<const __half*>(Bh), static_cast<const __half*>(Bl),
                                                      wcol, C, L, T, twoF, row_slot, fix);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  TemporalBatch bt;
  bt.n = 1;
  bt.A[0] = h;
  bt.C[0] = C;
  bt.L[0] = L;
  bt.tile_start[0] = 0;
  bt.tile_start[1] = 0;
  return launch_gather(bt, Bh, Bl, wcol, T, twoF, L, fix, row_slot, s);
}

cudaError_t launch_temporal_tc_gather(const TemporalBatch& bt, const void* Bh, const void* Bl, const float* wcol,
                                      int T, int twoF, const TemporalFix& fix, cudaStream_t s) {
  if (T % 8 != 0 || bt.n < 1 || bt.n > kMaxBatch) return cudaErrorInvalidValue;
  const cudaError_t e = configure();
  if (e != cudaSuccess) return e;
  long long rows = 0;
  for (int b = 0; b < bt.n; ++b) rows += bt.L[b];
  return launch_gather(bt, Bh, Bl, wcol, T, twoF, (int)std::min<long long>(rows, 1LL << 30), fix, nullptr, s);
}

cudaError_t launch_temporal_tc_batched(const TemporalBatch& bt, const void* Bh, const void* Bl, const float* wcol,
                                       int T, int twoF, const TemporalFix& fix, int* counter, cudaStream_t s) {
  if (T % 8 != 0 || bt.n < 1 || bt.n > kMaxBatch) return cudaErrorInvalidValue;
  cudaError_t e = configure();
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int tiles = bt.tile_start[bt.n];
  const int grid = std::max(1, std::min(tiles, 2 * sm_count()));
  temporal_tc_batched_kernel<<<grid, NT, sizeof(TcSmem), s>>>(bt, static_cast<const __half*>(Bh),
                                                               static_cast<const __half*>(Bl), wcol, T, twoF, counter,
                                                               fix);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  long long rows = 0;
  for (int b = 0; b < bt.n; ++b) rows += bt.L[b];
  return launch_gather(bt, Bh, Bl, wcol, T, twoF, (int)std::min<long long>(rows, 1LL << 30), fix, nullptr, s);
}

}  // namespace nursd
