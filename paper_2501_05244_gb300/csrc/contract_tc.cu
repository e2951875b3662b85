// Transfer-function contraction of one reconstruction on the 5th-generation tensor cores (step a6,
// Eq. RSD_conv summed over frequency; and its adjoint, step a10).
//
// For symmetry class c with members s < 8 (the modes (+-p, +-q), (+-q, +-p)), table block
// A_c [R][I] (row r, inner index i) and input rows X[mode][I]:
//   plain:      out[mode(c, s)][r] = sum_i A_c[r][i] X[mode(c, s)][i]
//   conjugate:  out[mode(c, s)][r] = sum_i conj(A_c[r][i]) X[mode(c, s)][i]
// The forward is the plain form on the transposed table GcT [c][z][f] (r = z, i = f, X = U);
// the adjoint is the conjugate form on Gc [c][f][z] (r = f, i = z, X = Y).
//
// Complex as real, K = 2I with k = 2i + h (h = 0 real, 1 imaginary part): row r of A_c read as
// floats is exactly A[r][k], so the table streams into the MMA as stored.  B has N = 16 rows,
// n = 2s + o (o = 0 real, 1 imaginary part of the output), x = X[mode(c, s)][i] = (a, b):
//   plain:     B[2s][2i..2i+1] = (a, -b),  B[2s+1][2i..2i+1] = (b, a)
//   conjugate: B[2s][2i..2i+1] = (a,  b),  B[2s+1][2i..2i+1] = (b, -a)
// so D[r][2s] and D[r][2s+1] are the real and imaginary parts of out[mode(c, s)][r]: one
// M = 128, N = 16, K = 2I product per class.
//
// FP32 accuracy from tf32 products: x = x_hi + x_lo with x_hi = tf32(x) (round to nearest) and
// x_lo = x - x_hi; D = A_hi [B_hi | B_lo] + A_lo B_hi, the first as one N = 32 product whose
// second half the epilogue adds to the first.  Only A_lo B_lo (about 2^-22 of each product) and
// the tf32 rounding of the tails (about 2^-23) are missed.
//
// Data path per 16-element block of i (a K chunk of 32 floats):
//   - the table's 128 x 32-float box arrives by TMA (128-byte swizzle) in a ring of kTcStages slots;
//   - four "split" warps (one per 32-row quarter) read their rows, form head and tail, and write
//     both into tensor memory with tcgen05.st (the A operand of tcgen05.mma may sit in tensor
//     memory), so the table crosses shared memory once;
//   - the class's 8 input rows arrive by cp.async.bulk, and a builder warp forms the chunk's B tile
//     (32 rows: heads, then tails) in the 128-byte-swizzled K-major layout;
//   - one thread issues the MMAs; four epilogue warps read the class's accumulator (row r per
//     thread) and store out rows as 256-byte runs.
// Two split groups take alternate chunks.  Every mbarrier wait is bounded: on time-out the waiting
// role sets the CTA's abort flag and status bit 2, every role stops, the copy issuers wait
// (bounded) for their copies in flight, the MMA thread for its MMAs, and tensor memory is released
// after a final CTA barrier.
//
// Measured at 65,536 samples -> 256^2 x 128 voxels, F = 128 (M = 512, 33,153 classes): 1.04 ms for
// the forward and for the adjoint, against 0.83 and 0.85 ms for the FP32 bulk-copy kernel; the same
// data path without the MMAs takes 0.77 ms, and neither four independent accumulators, seven A
// slots nor an A head read straight from the TMA tile in shared memory helped.  At N = 16 and 32
// an MMA costs far more than its arithmetic, and a class offers 64 of them per 128 KB of table.
// Plans therefore run this form only when asked (NURSD_TUNE_CONTRACT_TC).
#include <cuda.h>

#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int kTcRows = 128;             // M: rows of a class block
constexpr int kTcChunk = 16;             // complex inner values per K chunk (32 floats, 128 bytes)
constexpr int kTcStages = 10;            // table boxes in flight (16 KB each)
constexpr int kTcA = 4;                  // A slots in tensor memory (64 columns each: head, tail)
constexpr int kTcB = 6;                  // B tiles (4 KB each)
constexpr int kTcU = 3;                  // input-row stages (8 rows each)
constexpr int kTcBox = kTcRows * 128;    // bytes of one table box
constexpr int kTcBTile = 32 * 128;       // bytes of one B tile
constexpr int kTcThreads = 16 * 32;
constexpr int kWarpTma = 0, kWarpMma = 1, kWarpBuild = 2, kWarpAlloc = 3, kWarpEpi = 4, kWarpSplit = 8;
constexpr uint32_t kTcCols = 512;        // tensor memory: 2 accumulators x 32, then kTcA x 64
constexpr long long kTcSpin = 1LL << 22;

struct TcCtl {
  unsigned long long raw_full[kTcStages], raw_empty[kTcStages];
  unsigned long long a_full[kTcA], a_empty[kTcA];
  unsigned long long b_full[kTcB], b_empty[kTcB];
  unsigned long long u_full[kTcU];
  unsigned long long acc_full[2], acc_empty[2], drain;
  unsigned tmem;
  int abort;
};
static_assert(sizeof(TcCtl) <= 1024, "control block exceeds the shared memory reserved for it");

__device__ __forceinline__ uint32_t tsa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(tsa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void tbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tsa(b)) : "memory");
}
__device__ __forceinline__ void tbar_expect(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tsa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool tbar_try(unsigned long long* b, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(tsa(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait; gives up early once another role aborted, and raises the flag on its own time-out.
__device__ __forceinline__ bool tbar_wait(unsigned long long* b, unsigned parity, volatile int* abort) {
  for (long long i = 0; i < kTcSpin; ++i) {
    if (tbar_try(b, parity)) return true;
    if ((i & 255) == 255 && *abort) return false;
  }
  *abort = 1;
  return false;
}
// Bounded wait for a copy or MMA already in flight (used while tearing down: no early exit).
__device__ __forceinline__ void tbar_drain(unsigned long long* b, unsigned parity) {
  for (long long i = 0; i < kTcSpin; ++i)
    if (tbar_try(b, parity)) return;
}
__device__ __forceinline__ void tfence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tfence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle layout (rows of 128
// bytes whose 16-byte chunks are XOR-permuted by row mod 8, 8-row groups 1024 bytes apart, tile
// base 1024-byte aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::tf32: tf32 A and B (K-major), fp32 D, M x N.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (tensor memory) (+)= A (tensor memory) x B (shared memory descriptor).
__device__ __forceinline__ void umma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(tsa(b))
               : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(x));
  return h;
}
__device__ __forceinline__ float tf32_rest(float x, uint32_t h) { return x - __uint_as_float(h); }

// Mode index ky*M + kx of member s (s < 8) of class (p, q): (+-p, +-q), (+-q, +-p); mode k is stored
// at index k + M/2 (M a power of two; +M/2 wraps onto -M/2).
__device__ __forceinline__ unsigned tc_member(int p, int q, int s, int M) {
  const int a = (s < 4) ? p : q, b = (s < 4) ? q : p;
  const int kx = (s & 1) ? -a : a, ky = (s & 2) ? -b : b;
  return (unsigned)(((ky + M / 2) & (M - 1)) * M + ((kx + M / 2) & (M - 1)));
}

struct TcArgs {
  const float2* X;     // input rows [M*M][I]
  const int2* cls_pq;  // (p, q) of each class
  int ncls, M, I;      // classes, grid size, inner length (complex)
  float2* out;         // output rows [M*M][kTcRows]
  int* status;
};

template <bool CONJ>
__global__ void __launch_bounds__(kTcThreads, 1) contract_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                    const TcArgs a) {
  extern __shared__ unsigned char raw_smem[];
  const uint32_t raw_addr = tsa(raw_smem);
  unsigned char* base = raw_smem + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  unsigned char* ring = base;                                 // kTcStages table boxes
  unsigned char* btile = ring + kTcStages * kTcBox;           // kTcB B tiles
  float2* ustage = reinterpret_cast<float2*>(btile + kTcB * kTcBTile);  // kTcU x [8][I]
  const int I = a.I, nk = I / kTcChunk;
  TcCtl& ctl = *reinterpret_cast<TcCtl*>(reinterpret_cast<unsigned char*>(ustage) + (size_t)kTcU * 8 * I * 8);
  volatile int* abort = &ctl.abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my_cls = (int)blockIdx.x < a.ncls ? (a.ncls - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int my_chunks = my_cls * nk;
  auto cls_of = [&](int j) { return (int)blockIdx.x + j * (int)gridDim.x; };

  if (threadIdx.x == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      tbar_init(&ctl.raw_full[i], 1);
      tbar_init(&ctl.raw_empty[i], 4);
    }
    for (int i = 0; i < kTcA; ++i) {
      tbar_init(&ctl.a_full[i], 4);
      tbar_init(&ctl.a_empty[i], 1);
    }
    for (int i = 0; i < kTcB; ++i) {
      tbar_init(&ctl.b_full[i], 1);
      tbar_init(&ctl.b_empty[i], 1);
    }
    for (int i = 0; i < kTcU; ++i) tbar_init(&ctl.u_full[i], 1);
    for (int i = 0; i < 2; ++i) {
      tbar_init(&ctl.acc_full[i], 1);
      tbar_init(&ctl.acc_empty[i], 4);
    }
    tbar_init(&ctl.drain, 1);
    ctl.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == kWarpAlloc) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tsa(&ctl.tmem)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    tfence_before();
  }
  __syncthreads();
  tfence_after();
  const uint32_t tmem = ctl.tmem;
  auto acc_col = [](int ab) { return (uint32_t)(ab * 32); };
  auto a_col = [](int slot) { return (uint32_t)(64 + slot * 64); };

  if (warp == kWarpTma) {
    // ---------------------------------------------------------------- table boxes by TMA
    if (lane == 0) {
      int g = 0;
      for (; g < my_chunks; ++g) {
        const int st = g % kTcStages;
        if (!tbar_wait(&ctl.raw_empty[st], ((g / kTcStages) & 1) ^ 1, abort)) break;
        const int c = cls_of(g / nk), kk = g - (g / nk) * nk;
        tbar_expect(&ctl.raw_full[st], kTcBox);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];\n" ::"r"(tsa(ring + st * kTcBox)),
            "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(kk * 2 * kTcChunk), "r"(c * kTcRows),
            "r"(tsa(&ctl.raw_full[st]))
            : "memory");
      }
      // the last box of each slot may still be landing: wait for it before the CTA can exit
      for (int h = max(0, g - kTcStages); h < g; ++h) tbar_drain(&ctl.raw_full[h % kTcStages], (h / kTcStages) & 1);
    }
  } else if (warp == kWarpBuild) {
    // ---------------------------------------------------------------- input rows and B tiles
    // the class's 8 input rows by cp.async.bulk (I * 8 bytes each), kTcU - 1 classes ahead; a stage
    // is reused only after this warp has built every tile from it
    const unsigned row_bytes = (unsigned)I * 8u;
    auto fetch = [&](int j) {
      if (lane == 0) {
        const int su = j % kTcU;
        const int2 pq = __ldg(a.cls_pq + cls_of(j));
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        tbar_expect(&ctl.u_full[su], 8u * row_bytes);
        for (int s = 0; s < 8; ++s)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                  tsa(ustage + ((size_t)su * 8 + s) * I)),
              "l"(a.X + (size_t)tc_member(pq.x, pq.y, s, a.M) * I), "r"(row_bytes), "r"(tsa(&ctl.u_full[su]))
              : "memory");
      }
    };
    int fetched = 0;
    for (; fetched < min(my_cls, kTcU - 1); ++fetched) fetch(fetched);
    const int s = lane >> 2, qq = lane & 3;  // member s, complex values 4 qq .. 4 qq + 3 of the chunk
    bool ok = true;
    int g = 0;
    for (int j = 0; j < my_cls && ok; ++j) {
      if (fetched < my_cls) fetch(fetched++);
      const int su = j % kTcU;
      if (!__all_sync(0xffffffffu, tbar_wait(&ctl.u_full[su], (j / kTcU) & 1, abort))) {
        ok = false;
        break;
      }
      const float2* xr = ustage + ((size_t)su * 8 + s) * I;
      for (int kk = 0; kk < nk; ++kk, ++g) {
        const int sb = g % kTcB;
        if (!__all_sync(0xffffffffu, tbar_wait(&ctl.b_empty[sb], ((g / kTcB) & 1) ^ 1, abort))) {
          ok = false;
          break;
        }
        const float4 x01 = *reinterpret_cast<const float4*>(xr + kk * kTcChunk + 4 * qq);
        const float4 x23 = *reinterpret_cast<const float4*>(xr + kk * kTcChunk + 4 * qq + 2);
        const float av[4] = {x01.x, x01.z, x23.x, x23.z}, bv[4] = {x01.y, x01.w, x23.y, x23.w};
        uint32_t ah[4], bh[4];
        float al[4], bl[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          ah[t] = tf32_rna(av[t]);
          al[t] = tf32_rest(av[t], ah[t]);
          bh[t] = tf32_rna(bv[t]);
          bl[t] = tf32_rest(bv[t], bh[t]);
        }
        const uint32_t sg = 0x80000000u;
        unsigned char* tile = btile + sb * kTcBTile;
        // row n, 16-byte chunk q of the swizzled tile
        auto put = [&](int n, int q, uint4 v) {
          *reinterpret_cast<uint4*>(tile + n * 128 + ((q ^ (n & 7)) << 4)) = v;
        };
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {  // complex values 2 hh, 2 hh + 1 of this lane: chunk 2 qq + hh
          const int t0 = 2 * hh, t1 = 2 * hh + 1, q = 2 * qq + hh;
          const uint32_t a0 = ah[t0], a1 = ah[t1], b0 = bh[t0], b1 = bh[t1];
          const uint32_t la0 = __float_as_uint(al[t0]), la1 = __float_as_uint(al[t1]);
          const uint32_t lb0 = __float_as_uint(bl[t0]), lb1 = __float_as_uint(bl[t1]);
          if (!CONJ) {  // (a, -b) and (b, a)
            put(2 * s, q, make_uint4(a0, b0 ^ sg, a1, b1 ^ sg));
            put(2 * s + 1, q, make_uint4(b0, a0, b1, a1));
            put(16 + 2 * s, q, make_uint4(la0, lb0 ^ sg, la1, lb1 ^ sg));
            put(17 + 2 * s, q, make_uint4(lb0, la0, lb1, la1));
          } else {  // (a, b) and (b, -a)
            put(2 * s, q, make_uint4(a0, b0, a1, b1));
            put(2 * s + 1, q, make_uint4(b0, a0 ^ sg, b1, a1 ^ sg));
            put(16 + 2 * s, q, make_uint4(la0, lb0, la1, lb1));
            put(17 + 2 * s, q, make_uint4(lb0, la0 ^ sg, lb1, la1 ^ sg));
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) tbar_arrive(&ctl.b_full[sb]);
      }
    }
    // copies still landing in stages this warp has not consumed
    if (lane == 0)
      for (int j = max(0, fetched - kTcU); j < fetched; ++j) tbar_drain(&ctl.u_full[j % kTcU], (j / kTcU) & 1);
  } else if (warp == kWarpMma) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t id32 = tc_idesc(kTcRows, 32), id16 = tc_idesc(kTcRows, 16);
      int g = 0;
      bool ok = true;
      for (int j = 0; j < my_cls && ok; ++j) {
        const int ab = j & 1;
        if (!tbar_wait(&ctl.acc_empty[ab], ((j >> 1) & 1) ^ 1, abort)) break;
        tfence_after();
        const uint32_t d = tmem + acc_col(ab);
        for (int kk = 0; kk < nk; ++kk, ++g) {
          const int sa_ = g % kTcA, sb = g % kTcB;
          if (!tbar_wait(&ctl.a_full[sa_], (g / kTcA) & 1, abort) || !tbar_wait(&ctl.b_full[sb], (g / kTcB) & 1, abort)) {
            ok = false;
            break;
          }
          tfence_after();
          const uint32_t ahd = tmem + a_col(sa_), atl = ahd + 32;
          const uint64_t bd = sw128_desc(tsa(btile + sb * kTcBTile));
#pragma unroll
          for (int t = 0; t < 4; ++t) {  // 8 tf32 = 32 bytes of K per instruction
            umma_ts(d, ahd + 8 * t, bd + (uint64_t)(2 * t), id32, (kk | t) != 0);  // A_hi [B_hi | B_lo]
            umma_ts(d, atl + 8 * t, bd + (uint64_t)(2 * t), id16, 1u);             // A_lo B_hi
          }
          tc_commit(&ctl.a_empty[sa_]);
          tc_commit(&ctl.b_empty[sb]);
        }
        if (ok) tc_commit(&ctl.acc_full[ab]);
      }
      // every MMA issued has completed before the CTA tears down
      tc_commit(&ctl.drain);
      tbar_drain(&ctl.drain, 0);
    }
  } else if (warp >= kWarpSplit) {
    // ---------------------------------------------------------------- table rows -> tf32 head and tail in tensor memory
    const int grp = (warp - kWarpSplit) >> 2, quarter = warp & 3;
    const int r = quarter * 32 + lane;  // this thread's table row (tensor-memory lane)
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int g = grp; g < my_chunks; g += 2) {
      const int st = g % kTcStages;
      if (!__all_sync(0xffffffffu, tbar_wait(&ctl.raw_full[st], (g / kTcStages) & 1, abort))) break;
      const unsigned char* row = ring + st * kTcBox + r * 128;
      uint32_t hd[32], tl[32];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint4 v = *reinterpret_cast<const uint4*>(row + ((q ^ (r & 7)) << 4));
        hd[4 * q] = v.x;
        hd[4 * q + 1] = v.y;
        hd[4 * q + 2] = v.z;
        hd[4 * q + 3] = v.w;
      }
      __syncwarp();
      if (lane == 0) tbar_arrive(&ctl.raw_empty[st]);
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float x = __uint_as_float(hd[k]);
        hd[k] = tf32_rna(x);
        tl[k] = __float_as_uint(tf32_rest(x, hd[k]));
      }
      const int sa_ = g % kTcA;
      if (!__all_sync(0xffffffffu, tbar_wait(&ctl.a_empty[sa_], ((g / kTcA) & 1) ^ 1, abort))) break;
      tfence_after();
      tmem_st32(lane_base + a_col(sa_), hd);
      tmem_st32(lane_base + a_col(sa_) + 32, tl);
      asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
      tfence_before();
      __syncwarp();
      if (lane == 0) tbar_arrive(&ctl.a_full[sa_]);
    }
  } else if (warp >= kWarpEpi) {
    // ---------------------------------------------------------------- epilogue
    const int quarter = warp & 3, r = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int j = 0; j < my_cls; ++j) {
      const int ab = j & 1;
      if (!__all_sync(0xffffffffu, tbar_wait(&ctl.acc_full[ab], (j >> 1) & 1, abort))) break;
      tfence_after();
      uint32_t v[32];
      tmem_ld32(lane_base + acc_col(ab), v);
      tfence_before();
      __syncwarp();
      if (lane == 0) tbar_arrive(&ctl.acc_empty[ab]);
      const int2 pq = __ldg(a.cls_pq + cls_of(j));
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const float re = __uint_as_float(v[2 * s]) + __uint_as_float(v[16 + 2 * s]);
        const float im = __uint_as_float(v[2 * s + 1]) + __uint_as_float(v[17 + 2 * s]);
        a.out[(size_t)tc_member(pq.x, pq.y, s, a.M) * kTcRows + r] = make_float2(re, im);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && ctl.abort) atomicOr(a.status, 2);
  if (warp == kWarpAlloc) {
    tfence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols) : "memory");
  }
}

using TcEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TcEncodeFn tc_encode_fn() {
  static TcEncodeFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<TcEncodeFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

size_t tc_smem(int I) {
  return 1024 + (size_t)kTcStages * kTcBox + (size_t)kTcB * kTcBTile + (size_t)kTcU * 8 * I * 8 + 1024;
}

template <bool CONJ>
cudaError_t launch_tc(const CUtensorMap& map, const TcArgs& a, cudaStream_t s) {
  static int sms = 0;
  static size_t configured = 0;
  const size_t smem = tc_smem(a.I);
  if (configured < smem) {
    const cudaError_t e =
        cudaFuncSetAttribute(contract_tc_kernel<CONJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const int grid = std::min(a.ncls, sms);
  contract_tc_kernel<CONJ><<<grid, kTcThreads, smem, s>>>(map, a);
  return cudaGetLastError();
}

}  // namespace

bool contract_tc_supported(int M, int rows, int inner) {
  return M >= 2 && (M & (M - 1)) == 0 && rows == kTcRows && inner >= kTcChunk && inner % kTcChunk == 0 &&
         tc_smem(inner) <= 227 * 1024;
}

cudaError_t launch_contract_tc(const float2* X, const float2* table, const int2* cls_pq, int ncls, int M, int rows,
                               int inner, bool conj, float2* out, cudaStream_t s, int* status) {
  if (!contract_tc_supported(M, rows, inner) || ncls < 1 || !status || !X || !table || !cls_pq || !out ||
      reinterpret_cast<uintptr_t>(X) % 16 != 0 || reinterpret_cast<uintptr_t>(table) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(out) % 8 != 0)
    return cudaErrorInvalidValue;
  TcEncodeFn fn = tc_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  // the table as [ncls * rows] rows of 2 * inner floats, 32 x 128 boxes in the 128-byte swizzle
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * inner), (cuuint64_t)ncls * (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * kTcChunk), (cuuint32_t)kTcRows};
  const cuuint32_t estr[2] = {1, 1};
  if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2*>(table), dims, strides, box, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const TcArgs a{X, cls_pq, ncls, M, inner, out, status};
  return conj ? launch_tc<true>(map, a, s) : launch_tc<false>(map, a, s);
}

}  // namespace nursd
