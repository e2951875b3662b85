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
#include <algorithm>

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

// ------------------------------------------------------------------ bulk-copy form
// Same sums, persistent: warp w of the grid takes the units w, w + W, w + 2W, ...
// (W = warps in the grid; unit = class x column of 32 ZPL outputs x batch item,
// batch item fastest so a class's table block is re-read from L2 for the later
// items).  Each warp streams its units through a 3-stage shared-memory ring
// filled by cp.async.bulk (the TMA's 1-D mode) and completed on an mbarrier with
// a transaction count; the ring runs on across unit boundaries, so the next
// unit's rows are in flight while the current one finishes.  A stage holds
// kRows table rows (one contiguous copy of kRows x ZS values, or one per row when
// the column is narrower than the row); the class's 8 spectrum values of those rows
// come by plain loads, one per lane, issued as many stages ahead and held in
// registers until their stage is consumed.  Used when every column is full
// (J % (32 ZPL) == 0) and R % kRows == 0, so every copy is a whole number of
// 16-byte units.  Every
// barrier wait is bounded: on time-out the kernel sets status bit 2 and returns.
//
// Arithmetic: each spectrum value u is expanded once per stage to (ux, ux, -uy, uy)
// and acc += (ux, ux) * (gx, gy) + (-uy, uy) * (gy, gx) in two fma.rn.f32x2 per
// (output, member).  The conjugate form accumulates conj(u) g and conjugates the sum.
// Lane L holds outputs 2L, 2L + 1 (+ 64 k) of its column: 16-byte shared loads and
// global stores are contiguous across the warp.
constexpr int kTmaWarps = 16, kStages = 3, kRows = 4;
constexpr long long kWaitLimit = 1LL << 22;
// Bound (mbarrier polls) of the data waits of the bulk-copy form; the default unless a test shortens it
// (set_contract_wait_limit).  The drain after a time-out always uses kWaitLimit.
__device__ long long g_contract_wait_limit = kWaitLimit;

__device__ __forceinline__ unsigned sm_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sm_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sm_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   sm_addr(dst)),
               "l"(src), "r"(bytes), "r"(sm_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit = kWaitLimit) {
  for (long long it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(sm_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// d = a * b + c, lane-wise on two fp32 values, one instruction.
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
      " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}

template <int ZPL>
struct TmaShape {
  static constexpr int ZS = 32 * ZPL;
  static constexpr int kStageTable = kRows * ZS;  // float2
  static constexpr int kStage = kStageTable;
  static constexpr size_t kRingBytes = sizeof(float2) * kTmaWarps * kStages * kStage;
  static constexpr size_t kExpBytes = sizeof(float4) * kTmaWarps * 8 * kRows;  // expanded spectrum values
  static constexpr size_t kPtrBytes = sizeof(void*) * kTmaWarps * 9;            // producer's source rows
  static constexpr size_t kSmem =
      kRingBytes + kExpBytes + kPtrBytes + sizeof(unsigned long long) * kTmaWarps * kStages;
};

// Mode index ky*M + kx of member s (s < 8) of class (p, q): (+-p, +-q), (+-q, +-p).
__device__ __forceinline__ unsigned member_offset(int p, int q, int s, int M) {
  const int a = (s < 4) ? p : q, b = (s < 4) ? q : p;
  const int kx = (s & 1) ? -a : a, ky = (s & 2) ? -b : b;
  return (unsigned)(wrap_index(ky, M) * M + wrap_index(kx, M));
}

template <int ZPL, bool CONJ>
__global__ void __launch_bounds__(kTmaWarps * 32, 1) contract_tma_kernel(const float2* __restrict__ U,
                                                                      const float2* __restrict__ Gc,
                                                                      const int2* __restrict__ cls_pq, int ncls,
                                                                      int M, int F, int Z, float2* __restrict__ Y,
                                                                      long long u_stride, long long y_stride, int B,
                                                                      int* __restrict__ status) {
  using S = TmaShape<ZPL>;
  constexpr int ZS = S::ZS;
  extern __shared__ __align__(16) unsigned char raw[];
  pdl_wait();  // the spectra come from the kernel before
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* myring = reinterpret_cast<float2*>(raw) + (size_t)warp * kStages * S::kStage;
  float4* myexp = reinterpret_cast<float4*>(raw + S::kRingBytes) + warp * 8 * kRows;
  // producer's source rows of its current unit (each slot is written and read by one lane only):
  // slots 0..7 = the members' spectrum rows (lanes 0..7), slot 8 = the table column (lane 0)
  const float2** mysrc = reinterpret_cast<const float2**>(raw + S::kRingBytes + S::kExpBytes) + warp * 9;
  unsigned long long* mybar =
      reinterpret_cast<unsigned long long*>(raw + S::kRingBytes + S::kExpBytes + S::kPtrBytes) + warp * kStages;
  const int nz = Z / ZS, nchunk = F / kRows;
  const int nunit = ncls * nz * B;
  const int W = gridDim.x * kTmaWarps;
  const int w0 = blockIdx.x * kTmaWarps + warp;
  if (w0 >= nunit) return;  // whole warp; nothing below synchronises across warps

  // ---- producer: unit iu, chunk ich, ring sequence number seq; lane 0 copies the table rows,
  // every lane loads one member's spectrum value of the stage
  int iu = w0, ich = 0;
  float2 uring[kStages];  // spectrum values of the stages in flight, oldest first
  auto issue = [&](unsigned seq) {
    if (iu >= nunit) return;
    if (ich == 0) {
      const int b = iu % B, rest = iu / B;
      const int zc = rest % nz, c = rest / nz;
      const int2 pq = __ldg(cls_pq + c);
      if (lane < 8) mysrc[lane] = U + b * u_stride + (size_t)member_offset(pq.x, pq.y, lane, M) * F;
      if (lane == 0) mysrc[8] = Gc + (size_t)c * F * Z + (size_t)zc * ZS;
    }
    const int st = seq % kStages, f0 = ich * kRows;
    float2* dst = myring + st * S::kStage;
    if (lane == 0) mbar_expect(mybar + st, (unsigned)(sizeof(float2) * kRows * ZS));
    __syncwarp();
    if (lane == 0) {
      const float2* g = mysrc[8];
      if (ZS == Z) {  // the stage's rows are contiguous in the table
        bulk_g2s(dst, g + (size_t)f0 * Z, (unsigned)(sizeof(float2) * kRows * ZS), mybar + st);
      } else {
        for (int r = 0; r < kRows; ++r)
          bulk_g2s(dst + r * ZS, g + (size_t)(f0 + r) * Z, (unsigned)(sizeof(float2) * ZS), mybar + st);
      }
    }
    // lane s * kRows + r: member s's spectrum value at frequency f0 + r, into the register ring (eight
    // 32-byte bulk copies per stage would quadruple the copy operations the SM issues)
    uring[kStages - 1] = __ldg(mysrc[lane / kRows] + f0 + lane % kRows);
    if (++ich == nchunk) {
      ich = 0;
      iu += W;
    }
  };
  if (lane == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(mybar + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  auto rotate = [&] {
#pragma unroll
    for (int q = 0; q + 1 < kStages; ++q) uring[q] = uring[q + 1];
  };
  for (unsigned k = 0; k < kStages; ++k) {
    rotate();
    issue(k);
  }

  // ---- consumer
  unsigned cseq = 0;
  const int zl = 2 * lane;  // outputs zl, zl + 1 (+ 64 h, h < ZPL / 2) of the column
  bool ok = true;
  for (int cu = w0; cu < nunit && ok; cu += W) {
    float2 acc[ZPL][8];
#pragma unroll
    for (int i = 0; i < ZPL; ++i)
#pragma unroll
      for (int s = 0; s < 8; ++s) acc[i][s] = make_float2(0.f, 0.f);
    for (int ch = 0; ch < nchunk; ++ch) {
      const int st = cseq % kStages;
      // the bound is read at each wait (not held in a register across the loop)
      if (!mbar_wait(mybar + st, (cseq / kStages) & 1, *reinterpret_cast<volatile long long*>(&g_contract_wait_limit))) {
        ok = false;
        break;
      }
      const float2* stage = myring + st * S::kStage;
      {  // expand this stage's 8 x kRows spectrum values, one per lane
        const float2 u = uring[0];
        myexp[lane] = CONJ ? make_float4(u.x, u.x, u.y, -u.y) : make_float4(u.x, u.x, -u.y, u.y);
      }
      __syncwarp();
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        float2 gv[ZPL], gs[ZPL];
#pragma unroll
        for (int h = 0; h < ZPL / 2; ++h) {
          const float4 t = *reinterpret_cast<const float4*>(stage + r * ZS + 64 * h + zl);
          gv[2 * h] = make_float2(t.x, t.y);
          gv[2 * h + 1] = make_float2(t.z, t.w);
        }
#pragma unroll
        for (int i = 0; i < ZPL; ++i) gs[i] = make_float2(gv[i].y, gv[i].x);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const float4 e = myexp[s * kRows + r];
          const float2 uu = make_float2(e.x, e.y), vv = make_float2(e.z, e.w);
#pragma unroll
          for (int i = 0; i < ZPL; ++i) {
            acc[i][s] = pfma(uu, gv[i], acc[i][s]);
            acc[i][s] = pfma(vv, gs[i], acc[i][s]);
          }
        }
      }
      __syncwarp();  // every lane has read this stage and the expanded values
      rotate();
      issue(cseq + kStages);
      ++cseq;
    }
    if (!ok) break;
    const int b = cu % B, rest = cu / B;
    const int zc = rest % nz, c = rest / nz;
    const int2 pq = __ldg(cls_pq + c);
    const unsigned moff = member_offset(pq.x, pq.y, lane & 7, M);
    float2* yb = Y + b * y_stride + (size_t)zc * ZS + zl;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      float2* dst = yb + (size_t)__shfl_sync(0xffffffffu, moff, s) * Z;
#pragma unroll
      for (int h = 0; h < ZPL / 2; ++h) {
        const float2 a0 = acc[2 * h][s], a1 = acc[2 * h + 1][s];
        *reinterpret_cast<float4*>(dst + 64 * h) =
            CONJ ? make_float4(a0.x, -a0.y, a1.x, -a1.y) : make_float4(a0.x, a0.y, a1.x, a1.y);
      }
    }
  }
  if (!ok) {
    if (lane == 0) atomicOr(status, 2);
    // let this warp's copies in flight land (bounded) before the CTA's shared memory goes away
    for (int st = 0; st < kStages; ++st) {
      mbar_wait(mybar + st, 0);
      mbar_wait(mybar + st, 1);
    }
  }
}

}  // namespace

cudaError_t set_contract_wait_limit(long long polls, cudaStream_t s) {
  const long long v = polls >= 0 ? polls : kWaitLimit;
  return cudaMemcpyToSymbolAsync(g_contract_wait_limit, &v, sizeof(v), 0, cudaMemcpyHostToDevice, s);
}

namespace {

template <int ZPL, bool CONJ>
cudaError_t launch_tma(const float2* U, const float2* Gc, const int2* cls_pq, int ncls, int M, int F, int Z, float2* Y,
                       cudaStream_t s, int B, long long u_stride, long long y_stride, int* status) {
  constexpr int ZS = TmaShape<ZPL>::ZS;
  const size_t smem = TmaShape<ZPL>::kSmem;
  static bool configured = false;
  static int sms = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(contract_tma_kernel<ZPL, CONJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    configured = true;
  }
  const long long nunit = (long long)ncls * (Z / ZS) * B;
  if (nunit >= (1LL << 31)) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(sms, (nunit + kTmaWarps - 1) / kTmaWarps);
  return launch_pdl(contract_tma_kernel<ZPL, CONJ>, dim3(grid), dim3(kTmaWarps * 32), smem, s, U, Gc, cls_pq, ncls, M,
                    F, Z, Y, u_stride, y_stride, B, status);
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
                       float2* Out, cudaStream_t s, int* status) {
  if (R > 256) return cudaErrorInvalidValue;
  if (status && R % kRows == 0) {  // whole 16-byte copies and full CTA columns: the bulk-copy pipeline
    if (J % 128 == 0) return launch_tma<4, CONJ>(In, T, cls_pq, ncls, M, R, J, Out, s, 1, 0, 0, status);
    if (J == 64) return launch_tma<2, CONJ>(In, T, cls_pq, ncls, M, R, J, Out, s, 1, 0, 0, status);
  }
  // outputs per lane (a CTA column covers 32*ZPL of them): 4 for deep extents, fewer for shallow ones.
  if (J > 64) return launch_zpl<4, CONJ>(In, T, cls_pq, ncls, M, R, J, Out, s);
  if (J > 32) return launch_zpl<2, CONJ>(In, T, cls_pq, ncls, M, R, J, Out, s);
  return launch_zpl<1, CONJ>(In, T, cls_pq, ncls, M, R, J, Out, s);
}

}  // namespace

cudaError_t launch_contract(const float2* U, const float2* Gc, const int2* cls_pq, int ncls, int M, int F, int Z,
                            float2* Y, cudaStream_t s, int* status) {
  return launch_dir<false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s, status);
}

cudaError_t launch_contract_batched(const float2* U, long long u_stride, const float2* Gc, const int2* cls_pq,
                                   int ncls, int M, int F, int Z, float2* Y, long long y_stride, int B,
                                   cudaStream_t s, int* status) {
  if (F > 256 || B < 1) return cudaErrorInvalidValue;
  if (status && F % kRows == 0) {
    if (Z % 128 == 0) return launch_tma<4, false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s, B, u_stride, y_stride, status);
    if (Z == 64) return launch_tma<2, false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s, B, u_stride, y_stride, status);
  }
  if (Z > 64) return launch_zpl<4, false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s, B, u_stride, y_stride);
  if (Z > 32) return launch_zpl<2, false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s, B, u_stride, y_stride);
  return launch_zpl<1, false>(U, Gc, cls_pq, ncls, M, F, Z, Y, s, B, u_stride, y_stride);
}

cudaError_t launch_contract_adjoint(const float2* Yt, const float2* GcT, const int2* cls_pq, int ncls, int M, int F,
                                    int Z, float2* R, cudaStream_t s, int* status) {
  return launch_dir<true>(Yt, GcT, cls_pq, ncls, M, Z, F, R, s, status);
}

}  // namespace nursd
