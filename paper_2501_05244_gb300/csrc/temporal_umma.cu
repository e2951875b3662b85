// Temporal transform on the 5th-generation tensor cores (Eq. PF_Response with Eq. PFPacket):
// C[L][2F] = H[L][T] * B[T][2F] * diag(w), B[n][2f] = cos(w_f t_n), B[n][2f+1] = -sin(w_f t_n),
// as tcgen05.mma (kind::f16: fp16 operands, fp32 accumulation in tensor memory); the weight
// w_f of each column pair is applied in the epilogue, so B holds unit-modulus values only.
//
// FP32 accuracy from fp16 products, as in the mma.sync form: x = x_hi + x_lo with
// x_lo = fp16(x - x_hi), and C = H_hi B_hi + H_hi B_lo + H_lo B_hi, every product
// exact in the fp32 accumulator.  B's head and tail are split once at plan time
// ([2F][T], K-major); H is split as it is staged, and a K-block whose H_lo is all
// zero (photon counts below 2048 are exact in fp16) skips the H_lo product.
//
// FP32 range: the split keeps ~22 bits of every value of a row whose max |h| lies in
// [2^-3, 65504) (an error below 2^-22 of the row's max).  The H producers track each row's
// max; a row outside that window (a bin above fp16's range, or pre-normalised data) is listed
// with the exponent e that brings its max into [2^14, 2^15), and a second launch of this
// kernel in gather mode recomputes only the listed rows from h 2^-e (exact), multiplying the
// accumulator by 2^e in the epilogue.  With nothing listed that launch exits at once.
//
// One CTA per SM walks 128-row tiles of H (tile blockIdx.x + j gridDim.x).  Warp roles:
//   0-3  epilogue: tcgen05.ld of the 128 x 2F accumulator (one row per thread), fp32 stores
//        (row l to row row_slot[l] when a slot order is given);
//        two accumulators in tensor memory, so a tile's epilogue overlaps the next tile's MMAs
//   4-11 H producers: each K-block's 128 x 32 values of H (plain launch: from a ring of TMA
//        boxes; gather and batch launches: global loads six K-blocks ahead, ~96 KB per SM in
//        flight), fp16 head/tail split, stores into the 64-byte-swizzled K-major operand layout
//   12   B producer (one thread): TMA tiled copies of the 32 x 2F head and tail blocks
//   13   MMA issuer (one thread): 2 k-steps of 16 per K-block, tcgen05.commit to the
//        stage's "empty" barrier and, after the tile's last K-block, to the accumulator's
//        "full" barrier
//   14   H copier (plain launch, one thread): TMA tiled copies of H's 128 x 32 boxes (128-byte
//        swizzle, rows past L read as zero) into a ring of 5 to 8 slots
// Stages (K-blocks of 32; three in the plain launch, four otherwise) hold A_hi, A_lo (128 x 32
// fp16 each) and B_hi, B_lo (2F x 32 fp16 each), so the next twiddle copies start two or three
// K-blocks before they are needed.  In the plain launch the ring keeps 80 to 128 KB of H in flight
// per SM (at 65,536 x 1,024 samples: 0.110 ms against 0.123 ms for the load-based producers).
// Every mbarrier wait is bounded: on time-out the waiting role sets an abort flag (and
// status bit 4), every role stops issuing work, copies and MMAs in flight are drained,
// and tensor memory is released before the CTA exits.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {

namespace {

constexpr int kBM = 128, kBK = 32, kUStages = 4;
constexpr int kEpiWarps = 4, kCvtWarps = 8;
constexpr int kProducerWarp = kEpiWarps + kCvtWarps, kMmaWarp = kProducerWarp + 1, kHWarp = kMmaWarp + 1;
constexpr int kUThreads = (kHWarp + 1) * 32;
constexpr int kRawBox = kBM * kBK * 4;  // one box of H: 128 rows x 32 fp32 (16 KB)
constexpr int kRawMax = 8;
constexpr size_t kSmemMax = 232448;     // dynamic shared memory of one CTA
constexpr long long kUSpin = 1LL << 22;

template <int N2, int MODE>
struct UShape {
  static constexpr int kA = kBM * 64;  // one A tile: 128 rows x 32 fp16 (64-byte rows)
  static constexpr int kB = N2 * 64;   // one B tile: N2 rows x 32 fp16
  static constexpr int kStage = 2 * kA + 2 * kB;
  static constexpr int kAcc = N2 < 32 ? 32 : N2;  // tensor-memory columns per accumulator
  static constexpr bool kTma = MODE == 0;  // H by TMA boxes (plain launch)
  static constexpr int kNS = kTma ? 3 : kUStages;
  // 1 KB of alignment slack, the stages, the H ring (plain launch) and the control block.  Without
  // the ring, for N2 = 256 this stays within the 196 KB shared-memory carveout (a larger carveout
  // leaves too little L1 for the histogram loads); with it, as many 16 KB slots as fit (up to 8).
  static constexpr size_t kBase = 1024 + (size_t)kNS * kStage;
  static constexpr int kNR =
      kTma ? ((kSmemMax - 1536 - kBase) / kRawBox < kRawMax ? (int)((kSmemMax - 1536 - kBase) / kRawBox) : kRawMax)
           : 0;
  static constexpr size_t kSmem = kBase + (size_t)kNR * kRawBox + 1536;
  static_assert(!kTma || kNR >= 4, "the H ring needs at least four slots");
  static_assert(kSmem <= kSmemMax, "shared memory of one CTA exceeded");
};

struct Ctl {  // control block after the stages (at most the 1536 bytes the shape reserves)
  unsigned long long full_a[kUStages], full_b[kUStages], empty[kUStages];
  unsigned long long raw_full[kRawMax], raw_empty[kRawMax];  // H ring (plain launch)
  unsigned long long acc_full[2], acc_empty[2], drain;
  unsigned tmem;
  int abort;
  int lo[kUStages][kCvtWarps];
  // running max |h| of each producer thread's two rows (first launch): the upper 16 bits of the
  // FP32 magnitude rounded up, row q in bits 16 q .. 16 q + 15
  uint32_t rmax[kCvtWarps * 32];
  int listed;  // gather launch: rows listed by the first launch
};
static_assert(sizeof(Ctl) <= 1536, "control block exceeds the shared memory reserved for it");

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned long long* b, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(sa(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase of parity `parity`; gives up early once another role aborted.
__device__ __forceinline__ bool bar_wait(unsigned long long* b, unsigned parity, volatile int* abort) {
  for (long long i = 0; i < kUSpin; ++i) {
    if (bar_try(b, parity)) return true;
    if ((i & 255) == 255 && *abort) return false;
  }
  *abort = 1;
  return false;
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 64-byte swizzle layout
// (rows of 64 bytes whose 16-byte chunks are XOR-permuted by (row / 2) mod 4, 8-row groups
// 512 bytes apart, tile base 1024-byte aligned).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;                  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)4 << 61;                           // 64-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: fp16 A and B (K-major), fp32 D, M x N.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sa(b))
               : "memory");
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          sa(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sa(b))
      : "memory");
}

// 32 consecutive fp32 columns of this warp's 32 tensor-memory lanes (one per thread).
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

// fp16 head of two floats packed (low half = a), and the fp16 tail of what the head misses.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Per-item inputs of the batch mode: item b's H, C and row count, and its first 128-row tile
// (tile_start[n] = all tiles); nothing in the other modes.
template <int MODE>
struct UItems {};
template <>
struct UItems<2> {
  TemporalBatch bt;
};

// MODE 0: rows 0 .. L-1 of H; rows whose max |h| lies outside the split's window are listed in fix
// (as {row, e, 0, 0}).  MODE 2: the same for every item of a batch (tile t of item b is row block
// t - tile_start[b] of item b; listed as {row, e, b, 0}).  MODE 1 (gather): the listed rows
// (fix.list[0 .. *fix.count), each row index below
// L), scaled by 2^-e before the split and by 2^e in the epilogue.
template <int N2, int MODE>
__global__ void __launch_bounds__(kUThreads, 1) temporal_umma_kernel(const float* __restrict__ H,
                                                                     float* __restrict__ C, int L, int T,
                                                                     const __grid_constant__ CUtensorMap tm_hi,
                                                                     const __grid_constant__ CUtensorMap tm_lo,
                                                                     int* __restrict__ status,
                                                                     const int* __restrict__ row_slot,
                                                                     const float* __restrict__ wcol,
                                                                     const TemporalFix fix,
                                                                     const __grid_constant__ UItems<MODE> ui,
                                                                     const __grid_constant__ CUtensorMap tm_h) {
  constexpr bool GATHER = MODE == 1, BATCH = MODE == 2;
  using S = UShape<N2, MODE>;
  constexpr int NS = S::kNS;
  pdl_wait();  // the gather launch reads the list the plain launch before it wrote
  // the plain launch lets its dependent (the gather launch) start only at its end, so that launch's
  // CTAs never wait on SMs that the work beside this kernel (the relay-sample sort) runs on
  if constexpr (MODE != 0) pdl_trigger();
  extern __shared__ unsigned char raw[];
  const uint32_t raw_addr = sa(raw);
  unsigned char* base = raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  unsigned char* hring = base + NS * S::kStage;  // H boxes (plain launch)
  Ctl& ctl = *reinterpret_cast<Ctl*>(hring + S::kNR * kRawBox);
  if (GATHER) {
    if (threadIdx.x == 0) ctl.listed = temporal_fix_take(fix);
    __syncthreads();
  }
  const int nrows = GATHER ? min(ctl.listed, fix.cap) : L;
  int ntiles = (nrows + kBM - 1) / kBM;
  if constexpr (BATCH) ntiles = ui.bt.tile_start[ui.bt.n];
  const int nkb = T / kBK;
  const int kb_shift = (nkb & (nkb - 1)) == 0 ? __ffs(nkb) - 1 : -1;  // K-blocks per tile a power of two
  if (GATHER && (int)blockIdx.x >= ntiles) return;  // the whole CTA: nothing listed for it
  volatile int* abort = &ctl.abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int my_iters = my_tiles * nkb;
  auto a_hi = [&](int st) { return base + st * S::kStage; };
  auto a_lo = [&](int st) { return base + st * S::kStage + S::kA; };
  auto b_hi = [&](int st) { return base + st * S::kStage + 2 * S::kA; };
  auto b_lo = [&](int st) { return base + st * S::kStage + 2 * S::kA + S::kB; };
  // Batch mode: the item of tile t (tiles come in increasing order per role, so the search resumes
  // from the last item found) and its rows; other modes: item 0, H, C, L
  struct Src {
    int b, t0;  // item, its first tile
    const float* h;
    float* c;
    int L;
  };
  auto item_of = [&](int t, Src& sc) {
    if constexpr (BATCH) {
      int b = sc.b;
      while (b + 1 < ui.bt.n && t >= ui.bt.tile_start[b + 1]) ++b;
      sc.b = b;
      sc.t0 = ui.bt.tile_start[b];
      sc.h = ui.bt.A[b];
      sc.c = ui.bt.C[b];
      sc.L = ui.bt.L[b];
    } else {
      sc.b = 0;
      sc.t0 = 0;
      sc.h = H;
      sc.c = C;
      sc.L = L;
    }
  };
  // H row of position pos of the item (-1: none) and, in the gather launch, its exponent
  auto row_of = [&](int pos, int& x, int Lr) -> int {
    x = 0;
    if (!GATHER) return pos < Lr ? pos : -1;
    if (pos >= nrows) return -1;
    const int4 en = fix.list[pos];
    x = en.y;
    return (en.x >= 0 && en.x < L) ? en.x : -1;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      bar_init(&ctl.full_a[s], kCvtWarps);
      bar_init(&ctl.full_b[s], 1);
      bar_init(&ctl.empty[s], 1);
    }
    for (int s = 0; s < S::kNR; ++s) {
      bar_init(&ctl.raw_full[s], 1);
      bar_init(&ctl.raw_empty[s], kCvtWarps);
    }
    for (int s = 0; s < 2; ++s) {
      bar_init(&ctl.acc_full[s], 1);
      bar_init(&ctl.acc_empty[s], kEpiWarps);
    }
    bar_init(&ctl.drain, 1);
    ctl.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(&ctl.tmem)),
                 "r"(2 * S::kAcc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    fence_before_sync();
  }
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = ctl.tmem;

  if (warp < kEpiWarps) {
    // ---------------------------------------------------------------- epilogue
    Src esrc{0, 0, H, C, L};
    for (int j = 0; j < my_tiles; ++j) {
      const int ab = j & 1;
      if (!__all_sync(0xffffffffu, bar_wait(&ctl.acc_full[ab], (j >> 1) & 1, abort))) break;
      fence_after_sync();
      int x = 0;
      const int t = (int)blockIdx.x + j * (int)gridDim.x;
      item_of(t, esrc);
      int orow = row_of((t - esrc.t0) * kBM + warp * 32 + lane, x, esrc.L);
      if (orow >= 0 && row_slot) orow = __ldg(row_slot + orow);
      float* const Cb = esrc.c;
      const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ab * S::kAcc);
#pragma unroll 1
      for (int c0 = 0; c0 < N2; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tb + c0, r);
        if (orow >= 0) {
          float4* dst = reinterpret_cast<float4*>(Cb + (size_t)orow * N2 + c0);
          const float4* w4 = reinterpret_cast<const float4*>(wcol + c0);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 w = __ldg(w4 + q);
            float4 v = make_float4(__uint_as_float(r[4 * q]) * w.x, __uint_as_float(r[4 * q + 1]) * w.y,
                                   __uint_as_float(r[4 * q + 2]) * w.z, __uint_as_float(r[4 * q + 3]) * w.w);
            if (GATHER) {
              v.x = ldexpf(v.x, x);
              v.y = ldexpf(v.y, x);
              v.z = ldexpf(v.z, x);
              v.w = ldexpf(v.w, x);
            }
            dst[q] = v;
          }
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) bar_arrive(&ctl.acc_empty[ab]);
    }
  } else if (warp < kEpiWarps + kCvtWarps) {
    // ---------------------------------------------------------------- H producers
    const int cw = warp - kEpiWarps, ct = cw * 32 + lane;
    // task q < 2 of a K-block: row ct / 4 + 64 q of the tile, 16-byte chunk ct % 4 (8 consecutive K values)
    const int r0 = ct >> 2, ch = ct & 3;
    uint32_t* rmax = ctl.rmax + ct;  // this thread's two rows' running max over the tile's K-blocks
    // a register set holds K-blocks 2 p and 2 p + 1 (4 float4 each)
    Src lsrc{0, 0, H, C, L}, ssrc{0, 0, H, C, L};  // the loads' and the staging's current item
    auto load = [&](float4 (&v)[8], int pr) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int it = 2 * pr + h;
        if (it >= my_iters) return;
        const int j = kb_shift >= 0 ? it >> kb_shift : it / nkb, kb = it - j * nkb;
        const int t = (int)blockIdx.x + j * (int)gridDim.x;
        item_of(t, lsrc);
        const int m0 = (t - lsrc.t0) * kBM;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          int x;
          const int row = row_of(m0 + r0 + 64 * q, x, lsrc.L);
          const float4* s4 = reinterpret_cast<const float4*>(lsrc.h + (size_t)max(row, 0) * T + kb * kBK + ch * 8);
          v[4 * h + 2 * q] = row >= 0 ? __ldg(s4) : make_float4(0.f, 0.f, 0.f, 0.f);
          v[4 * h + 2 * q + 1] = row >= 0 ? __ldg(s4 + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    };
    auto stage_one = [&](const float4* v, int it) -> bool {
      const int st = it % NS, ph = (it / NS) & 1;
      const int j = kb_shift >= 0 ? it >> kb_shift : it / nkb, kb = it - j * nkb;
      const int t = (int)blockIdx.x + j * (int)gridDim.x;
      item_of(t, ssrc);
      const int m0 = (t - ssrc.t0) * kBM;
      if (!__all_sync(0xffffffffu, bar_wait(&ctl.empty[st], ph ^ 1, abort))) return false;
      unsigned char* ah = a_hi(st);
      unsigned char* al = a_lo(st);
      uint32_t any = 0, mcode = 0;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int r = r0 + 64 * q;
        float4 x = v[2 * q], y = v[2 * q + 1];
        if (GATHER) {
          int e;
          row_of(m0 + r, e, ssrc.L);
          x = make_float4(ldexpf(x.x, -e), ldexpf(x.y, -e), ldexpf(x.z, -e), ldexpf(x.w, -e));
          y = make_float4(ldexpf(y.x, -e), ldexpf(y.y, -e), ldexpf(y.z, -e), ldexpf(y.w, -e));
        } else {
          const float m = fmaxf(fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))),
                                fmaxf(fmaxf(fabsf(y.x), fabsf(y.y)), fmaxf(fabsf(y.z), fabsf(y.w))));
          mcode |= ((__float_as_uint(m) + 0xffffu) >> 16) << (16 * q);  // rounded up: zero only for 0
        }
        uint4 h, l;
        split2(x.x, x.y, h.x, l.x);
        split2(x.z, x.w, h.y, l.y);
        split2(y.x, y.y, h.z, l.z);
        split2(y.z, y.w, h.w, l.w);
        any |= (l.x | l.y | l.z | l.w) & 0x7fff7fffu;
        const int off = r * 64 + ((ch ^ ((r >> 1) & 3)) << 4);
        *reinterpret_cast<uint4*>(ah + off) = h;
        *reinterpret_cast<uint4*>(al + off) = l;
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      const int warp_any = __any_sync(0xffffffffu, any != 0);
      __syncwarp();
      if (lane == 0) {
        ctl.lo[st][cw] = warp_any;
        bar_arrive(&ctl.full_a[st]);
      }
      if (!GATHER) {
        const uint32_t rm = kb == 0 ? mcode : __vmaxu2(*rmax, mcode);
        *rmax = rm;
        if (kb == nkb - 1) {  // the tile's rows are complete: the 4 lanes of a row agree on its max
          uint32_t m = rm;
          m = __vmaxu2(m, __shfl_xor_sync(0xffffffffu, m, 1));
          m = __vmaxu2(m, __shfl_xor_sync(0xffffffffu, m, 2));
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int row = m0 + r0 + 64 * q;
            if (ch == 0 && row < ssrc.L) {
              const int e = temporal_row_exponent(__uint_as_float(((m >> (16 * q)) & 0xffffu) << 16));
              if (e != kRowInRange) {
                const int slot = atomicAdd(fix.count, 1);
                if (slot < fix.cap) fix.list[slot] = make_int4(row, e, ssrc.b, 0);
              }
            }
          }
        }
      }
      return true;
    };
    auto stage = [&](const float4 (&v)[8], int pr) -> bool {
      const int it = 2 * pr;
      if (!stage_one(v, it)) return false;
      return it + 1 >= my_iters || stage_one(v + 4, it + 1);
    };
    if constexpr (S::kTma) {  // this thread's two rows' 32 bytes of each K-block's box
      for (int it = 0; it < my_iters; ++it) {
        const int rs = it % S::kNR;
        if (!__all_sync(0xffffffffu, bar_wait(&ctl.raw_full[rs], (it / S::kNR) & 1, abort))) break;
        const unsigned char* box = hring + rs * kRawBox;
        float4 v[4];
#pragma unroll
        for (int q = 0; q < 2; ++q) {  // row r: 128 bytes whose 16-byte chunks are XOR-permuted by r mod 8
          const int r = r0 + 64 * q;
          v[2 * q] = *reinterpret_cast<const float4*>(box + r * 128 + (((2 * ch) ^ (r & 7)) << 4));
          v[2 * q + 1] = *reinterpret_cast<const float4*>(box + r * 128 + (((2 * ch + 1) ^ (r & 7)) << 4));
        }
        __syncwarp();
        if (lane == 0) bar_arrive(&ctl.raw_empty[rs]);
        if (!stage_one(v, it)) break;
      }
    } else {
    // three register sets in rotation: six K-blocks (about 96 KB per SM) in flight
    const int npairs = (my_iters + 1) / 2;
    float4 va[8], vb[8], vc[8];
    load(va, 0);
    load(vb, 1);
    load(vc, 2);
    for (int pr = 0; pr < npairs; pr += 3) {
      if (!stage(va, pr)) break;
      load(va, pr + 3);
      if (pr + 1 >= npairs || !stage(vb, pr + 1)) break;
      load(vb, pr + 4);
      if (pr + 2 >= npairs || !stage(vc, pr + 2)) break;
      load(vc, pr + 5);
    }
    }
  } else if (warp == kProducerWarp) {
    // ---------------------------------------------------------------- B producer
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < my_iters; ++it) {
        const int kb = it % nkb, st = it % NS, ph = (it / NS) & 1;
        if (!bar_wait(&ctl.empty[st], ph ^ 1, abort)) break;
        bar_expect_tx(&ctl.full_b[st], (unsigned)(2 * S::kB));
        tma_2d(b_hi(st), &tm_hi, kb * kBK, 0, &ctl.full_b[st]);
        tma_2d(b_lo(st), &tm_lo, kb * kBK, 0, &ctl.full_b[st]);
        issued = it + 1;
      }
      // the last copies have landed before the CTA can exit (already true unless a role aborted)
      for (int it = max(0, issued - NS); it < issued; ++it) {
        for (long long i = 0; i < kUSpin; ++i)
          if (bar_try(&ctl.full_b[it % NS], (it / NS) & 1)) break;
      }
    }
  } else if (warp == kHWarp) {
    // ---------------------------------------------------------------- H copier (plain launch)
    if constexpr (S::kTma) {
      if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < my_iters; ++it) {
        const int rs = it % S::kNR;
        if (!bar_wait(&ctl.raw_empty[rs], ((it / S::kNR) & 1) ^ 1, abort)) break;
        const int j = kb_shift >= 0 ? it >> kb_shift : it / nkb, kb = it - j * nkb;
        const int t = (int)blockIdx.x + j * (int)gridDim.x;
        bar_expect_tx(&ctl.raw_full[rs], (unsigned)kRawBox);
        tma_2d(hring + rs * kRawBox, &tm_h, kb * kBK, t * kBM, &ctl.raw_full[rs]);
        issued = it + 1;
      }
      // the last boxes have landed before the CTA can exit (already true unless a role aborted)
      for (int it = max(0, issued - S::kNR); it < issued; ++it)
        for (long long i = 0; i < kUSpin; ++i)
          if (bar_try(&ctl.raw_full[it % S::kNR], (it / S::kNR) & 1)) break;
      }
    }
  } else {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = f16_idesc(kBM, N2);
      int it = 0;
      bool ok = true;
      for (int j = 0; j < my_tiles && ok; ++j) {
        const int ab = j & 1;
        if (!bar_wait(&ctl.acc_empty[ab], ((j >> 1) & 1) ^ 1, abort)) break;
        fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(ab * S::kAcc);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int st = it % NS, ph = (it / NS) & 1;
          if (!bar_wait(&ctl.full_b[st], ph, abort) || !bar_wait(&ctl.full_a[st], ph, abort)) {
            ok = false;
            break;
          }
          fence_after_sync();
          int lo = 0;
#pragma unroll
          for (int w = 0; w < kCvtWarps; ++w) lo |= ctl.lo[st][w];
          const uint64_t dah = sw64_desc(sa(a_hi(st))), dal = sw64_desc(sa(a_lo(st)));
          const uint64_t dbh = sw64_desc(sa(b_hi(st))), dbl = sw64_desc(sa(b_lo(st)));
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {  // 16 fp16 = 32 bytes along K per instruction
            const uint64_t adv = (uint64_t)(2 * kk);
            umma_f16(d, dah + adv, dbh + adv, idesc, (kb | kk) != 0);
            umma_f16(d, dah + adv, dbl + adv, idesc, 1u);
            if (lo) umma_f16(d, dal + adv, dbh + adv, idesc, 1u);
          }
          umma_commit(&ctl.empty[st]);
        }
        if (ok) umma_commit(&ctl.acc_full[ab]);
      }
      // every MMA issued has completed before the CTA tears down
      umma_commit(&ctl.drain);
      for (long long i = 0; i < kUSpin; ++i)
        if (bar_try(&ctl.drain, 0)) break;
    }
  }
  __syncthreads();
  if constexpr (MODE == 0) pdl_trigger();
  if (threadIdx.x == 0 && ctl.abort) atomicOr(status, 4);
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * S::kAcc)
                 : "memory");
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// [rows][T] fp16, K-major, 32 x rows boxes in the 64-byte swizzle.
bool encode_b(CUtensorMap* m, const void* ptr, int T, int rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)T, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)T * sizeof(__half)};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N2, int MODE>
cudaError_t configure_n() {
  static bool configured = false;
  if (configured) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(temporal_umma_kernel<N2, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)UShape<N2, MODE>::kSmem);
  if (e == cudaSuccess) configured = true;
  return e;
}

// H [L][T] fp32 as 32 x 128 boxes in the 128-byte swizzle (rows past L read as zero).
bool encode_h(CUtensorMap* m, const float* h, int L, int T) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)T, (cuuint64_t)L};
  const cuuint64_t strides[1] = {(cuuint64_t)T * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(h), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N2>
cudaError_t launch_n(const TemporalMaps& m, const float* h, const float* wcol, float* C, int L, int T,
                     const TemporalFix& fix, int* status, cudaStream_t s, const int* row_slot) {
  using S0 = UShape<N2, 0>;
  using S1 = UShape<N2, 1>;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  cudaError_t e = configure_n<N2, 0>();
  if (e == cudaSuccess) e = configure_n<N2, 1>();
  if (e != cudaSuccess) return e;
  const int ntiles = (L + kBM - 1) / kBM;
  // the fewest CTAs with the same most tiles per CTA (the critical path): the SMs left over run the
  // work queued beside the transform (the relay-sample sort of a reconstruction)
  const int per_cta = (ntiles + sms - 1) / sms, grid = (ntiles + per_cta - 1) / per_cta;
  CUtensorMap tm_h;
  if (!encode_h(&tm_h, h, L, T)) return cudaErrorInvalidValue;
  e = launch_pdl(temporal_umma_kernel<N2, 0>, dim3(grid), dim3(kUThreads), S0::kSmem, s, h, C, L, T, m.hi, m.lo, status,
                 row_slot, wcol, fix, UItems<0>{}, tm_h);
  if (e != cudaSuccess) return e;
  // listed rows: at most min(L, cap); CTAs beyond the listed tiles return at once
  const int gtiles = (std::min(L, fix.cap) + kBM - 1) / kBM;
  if (gtiles <= 0) return cudaSuccess;
  return launch_pdl(temporal_umma_kernel<N2, 1>, dim3(std::min(gtiles, sms)), dim3(kUThreads), S1::kSmem, s, h, C, L,
                    T, m.hi, m.lo, status, row_slot, wcol, fix, UItems<1>{}, tm_h);
}

// Batch mode: bt.tile_start counts 128-row tiles.  The listed rows of every item are then
// recomputed by the mma.sync form's gather launch (temporal_tc.cu).
template <int N2>
cudaError_t launch_batch_n(const TemporalMaps& m, const TemporalBatch& bt, const float* wcol, int T,
                           const TemporalFix& fix, int* status, cudaStream_t s) {
  using S = UShape<N2, 2>;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  const cudaError_t e = configure_n<N2, 2>();
  if (e != cudaSuccess) return e;
  const int ntiles = bt.tile_start[bt.n];
  if (ntiles <= 0) return cudaSuccess;
  UItems<2> ui;
  ui.bt = bt;
  temporal_umma_kernel<N2, 2><<<std::min(ntiles, sms), kUThreads, S::kSmem, s>>>(nullptr, nullptr, 0, T, m.hi, m.lo,
                                                                                 status, nullptr, wcol, fix, ui,
                                                                                 CUtensorMap{});
  return cudaGetLastError();
}

}  // namespace

bool temporal_umma_supported(int T, int twoF) {
  return T > 0 && T % kBK == 0 && (twoF == 32 || twoF == 64 || twoF == 128 || twoF == 256);
}

bool make_temporal_maps(const void* Bh, const void* Bl, int T, int twoF, TemporalMaps* m) {
  m->ok = 0;
  if (!temporal_umma_supported(T, twoF)) return false;
  if (reinterpret_cast<uintptr_t>(Bh) % 16 != 0 || reinterpret_cast<uintptr_t>(Bl) % 16 != 0) return false;
  if (!encode_b(&m->hi, Bh, T, twoF) || !encode_b(&m->lo, Bl, T, twoF)) return false;
  m->ok = 1;
  return true;
}

cudaError_t launch_temporal_umma_batched(const TemporalMaps& m, const TemporalBatch& bt, const float* wcol, int T,
                                         int twoF, const TemporalFix& fix, int* status, cudaStream_t s) {
  if (!m.ok || !temporal_umma_supported(T, twoF) || bt.n < 1 || bt.n > kMaxBatch ||
      reinterpret_cast<uintptr_t>(wcol) % 16 != 0)
    return cudaErrorInvalidValue;
  for (int b = 0; b < bt.n; ++b) {
    if (bt.tile_start[b + 1] - bt.tile_start[b] != (bt.L[b] + kBM - 1) / kBM || bt.L[b] < 0)
      return cudaErrorInvalidValue;
    if (bt.L[b] > 0 && (reinterpret_cast<uintptr_t>(bt.A[b]) % 16 != 0 || reinterpret_cast<uintptr_t>(bt.C[b]) % 16 != 0))
      return cudaErrorInvalidValue;
  }
  switch (twoF) {
    case 32: return launch_batch_n<32>(m, bt, wcol, T, fix, status, s);
    case 64: return launch_batch_n<64>(m, bt, wcol, T, fix, status, s);
    case 128: return launch_batch_n<128>(m, bt, wcol, T, fix, status, s);
    default: return launch_batch_n<256>(m, bt, wcol, T, fix, status, s);
  }
}

cudaError_t launch_temporal_umma(const TemporalMaps& m, const float* h, const float* wcol, float* C, int L, int T,
                                 int twoF, const TemporalFix& fix, int* status, cudaStream_t s, const int* row_slot) {
  if (L <= 0) return cudaSuccess;
  if (!m.ok || !temporal_umma_supported(T, twoF) || reinterpret_cast<uintptr_t>(h) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(C) % 16 != 0 || reinterpret_cast<uintptr_t>(wcol) % 16 != 0)
    return cudaErrorInvalidValue;
  switch (twoF) {
    case 32: return launch_n<32>(m, h, wcol, C, L, T, fix, status, s, row_slot);
    case 64: return launch_n<64>(m, h, wcol, C, L, T, fix, status, s, row_slot);
    case 128: return launch_n<128>(m, h, wcol, C, L, T, fix, status, s, row_slot);
    default: return launch_n<256>(m, h, wcol, C, L, T, fix, status, s, row_slot);
  }
}

}  // namespace nursd
