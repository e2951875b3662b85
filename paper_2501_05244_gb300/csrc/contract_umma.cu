// Transfer-function contraction of a batch of reconstructions on the 5th-generation tensor cores.
//
// Items that share the plan's table make each symmetry class a dense product (Eq. RSD_conv summed
// over frequency, step a6): for class c with members s < 8 (the modes (+-p, +-q), (+-q, +-p)) and
// items b < B,
//   Y[b][mode(c, s)][z] = sum_f U[b][mode(c, s)][f] Gc[c][f][z],
// a (8 B) x F by F x Z complex product per class in which every table value is used 8 B times.
// Complex as real, rows r = (b, s) in tiles of 128 (16 items x 8 members):
//   D[r][n] = sum_k A[r][k] Bm[n][k],  k = 16 j + t over 8-frequency blocks j (f = 8 j + t mod 8),
//   A[r][16 j + t] = Re U[f] (t < 8), Im U[f] (t >= 8),
//   Bm[n][16 j + t] = n < Z: Re G[f][n] (t < 8), -Im G[f][n] (t >= 8);
//                     n >= Z: Im G[f][n - Z] (t < 8), Re G[f][n - Z] (t >= 8),
// so D[r][z] = Re Y and D[r][Z + z] = Im Y: one M = 128, N = 2Z, K = 2F product per tile as
// tcgen05.mma kind::tf32 with fp32 accumulation in tensor memory.
//
// FP32 accuracy from tf32 products: x = x_hi + x_lo with x_hi = tf32(x) (the top 10 explicit
// mantissa bits, round to nearest) and x_lo = tf32(x - x_hi), and D = A_hi B_hi + A_hi B_lo +
// A_lo B_hi, which misses only A_lo B_lo (about 2^-22 of each product).  tf32 keeps the FP32
// exponent range, so no scaling is needed.
//
// One CTA per SM walks the tiles (class-major, item blocks of 16 fastest, so a class's table
// block is read from L2 for its later item blocks).  Warp roles:
//   0-3   epilogue: tcgen05.ld of the 128 x 2Z accumulator (one row per thread), complex stores;
//         two accumulators, so a tile's epilogue overlaps the next tile's MMAs
//   4-11  producers: per 8-frequency block, the 128 rows' U values and the class's table rows
//         are loaded (five blocks ahead), split into tf32 head and tail and stored in the
//         64-byte-swizzled K-major operand layout
//   12    MMA issuer (one thread): per block two k-steps of 8 x 3 products, tcgen05.commit to the
//         stage's "empty" barrier, and after the tile's last block to the accumulator's "full"
// Every mbarrier wait is bounded: on time-out the waiting role sets the CTA's abort flag and
// status bit 2, every role stops, the MMA thread waits (bounded) for its MMAs and tensor memory
// is released after a final CTA barrier.
#include <algorithm>

#include "nursd_internal.cuh"

namespace nursd {
namespace {

constexpr int kCM = 128, kCStagesMax = 4;
constexpr int kCEpiWarps = 4, kCProdWarps = 8;
constexpr int kCMmaWarp = kCEpiWarps + kCProdWarps;
constexpr int kCThreads = (kCMmaWarp + 1) * 32;
constexpr long long kCSpin = 1LL << 22;
constexpr int kCAhead = 5;  // 8-frequency blocks of loads in flight per producer thread

template <int N2>
struct CShape {
  static constexpr int Z = N2 / 2;
  static constexpr int kStages = N2 <= 128 ? 4 : 3;
  static constexpr int kA = kCM * 64;  // one A tile: 128 rows x 16 tf32 (64-byte rows)
  static constexpr int kB = N2 * 64;   // one B tile: 2Z rows x 16 tf32
  static constexpr int kStage = 2 * kA + 2 * kB;
  static constexpr int kAcc = N2 < 32 ? 32 : N2;  // tensor-memory columns per accumulator
  static constexpr int kOut = kCEpiWarps * 32 * 33 * 8;  // epilogue transposes: 32 rows x 33 float2 per warp
  static constexpr size_t kSmem = 1024 + (size_t)kStages * kStage + kOut + 512;
};

struct CCtl {
  unsigned long long full[kCStagesMax], empty[kCStagesMax];
  unsigned long long acc_full[2], acc_empty[2], drain;
  unsigned tmem;
  int abort;
};
static_assert(sizeof(CCtl) <= 512, "control block exceeds the shared memory reserved for it");

__device__ __forceinline__ uint32_t csa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(csa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void cbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(csa(b)) : "memory");
}
__device__ __forceinline__ bool cbar_try(unsigned long long* b, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(csa(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait; gives up early once another role aborted, and raises the flag on its own time-out.
__device__ __forceinline__ bool cbar_wait(unsigned long long* b, unsigned parity, volatile int* abort) {
  for (long long i = 0; i < kCSpin; ++i) {
    if (cbar_try(b, parity)) return true;
    if ((i & 255) == 255 && *abort) return false;
  }
  *abort = 1;
  return false;
}
__device__ __forceinline__ void cfence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void cfence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile in the 64-byte swizzle layout (rows of 64
// bytes whose 16-byte chunks are XOR-permuted by (row / 2) mod 4, 8-row groups 512 bytes apart,
// tile base 1024-byte aligned).
__device__ __forceinline__ uint64_t csw64_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
// Instruction descriptor, kind::tf32: tf32 A and B (format code 2, K-major), fp32 D, M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void cumma_commit(unsigned long long* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(csa(b))
               : "memory");
}
__device__ __forceinline__ void ctmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
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

// tf32 head of x (round to nearest on the 13 dropped mantissa bits) and the tf32 tail of what it misses.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(x));
  uint32_t l;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(l) : "f"(x - __uint_as_float(h)));
  hi = h;
  lo = l;
}
__device__ __forceinline__ void split4(float a, float b, float c, float d, uint4& hi, uint4& lo) {
  split_tf32(a, hi.x, lo.x);
  split_tf32(b, hi.y, lo.y);
  split_tf32(c, hi.z, lo.z);
  split_tf32(d, hi.w, lo.w);
}

// Mode index ky*M + kx of member s (s < 8) of class (p, q): (+-p, +-q), (+-q, +-p).
__device__ __forceinline__ unsigned cmember(int p, int q, int s, int M) {
  const int a = (s < 4) ? p : q, b = (s < 4) ? q : p;
  const int kx = (s & 1) ? -a : a, ky = (s & 2) ? -b : b;
  // mode k is stored at index k + M/2 (M a power of two; +M/2 wraps onto -M/2)
  return (unsigned)(((ky + M / 2) & (M - 1)) * M + ((kx + M / 2) & (M - 1)));
}

// Y[b][mode][z] (row b at y_stride, mode rows of Z values) for every class and item b < B.
template <int N2>
__global__ void __launch_bounds__(kCThreads, 1) contract_umma_kernel(const float2* __restrict__ U, long long u_stride,
                                                                     const float2* __restrict__ Gc,
                                                                     const int2* __restrict__ cls_pq, int ncls, int M,
                                                                     int F, float2* __restrict__ Y,
                                                                     long long y_stride, int B,
                                                                     int* __restrict__ status) {
  using S = CShape<N2>;
  constexpr int Z = S::Z, NS = S::kStages;
  extern __shared__ unsigned char raw[];
  const uint32_t raw_addr = csa(raw);
  unsigned char* base = raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
  float2* obuf = reinterpret_cast<float2*>(base + NS * S::kStage);  // [4 warps][32 rows][33]
  CCtl& ctl = *reinterpret_cast<CCtl*>(base + NS * S::kStage + S::kOut);
  volatile int* abort = &ctl.abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nib = (B + 15) / 16;  // item blocks of 16 per class
  const int ntiles = ncls * nib, nkb = F / 8;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int my_iters = my_tiles * nkb;
  auto a_hi = [&](int st) { return base + st * S::kStage; };
  auto a_lo = [&](int st) { return base + st * S::kStage + S::kA; };
  auto b_hi = [&](int st) { return base + st * S::kStage + 2 * S::kA; };
  auto b_lo = [&](int st) { return base + st * S::kStage + 2 * S::kA + S::kB; };

  if (threadIdx.x == 0) {
    for (int st = 0; st < NS; ++st) {
      cbar_init(&ctl.full[st], kCProdWarps);
      cbar_init(&ctl.empty[st], 1);
    }
    for (int i = 0; i < 2; ++i) {
      cbar_init(&ctl.acc_full[i], 1);
      cbar_init(&ctl.acc_empty[i], kCEpiWarps);
    }
    cbar_init(&ctl.drain, 1);
    ctl.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(csa(&ctl.tmem)),
                 "r"(2 * S::kAcc)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    cfence_before();
  }
  __syncthreads();
  cfence_after();
  const uint32_t tmem = ctl.tmem;

  if (warp < kCEpiWarps) {
    // ---------------------------------------------------------------- epilogue
    for (int j = 0; j < my_tiles; ++j) {
      const int ab = j & 1;
      if (!__all_sync(0xffffffffu, cbar_wait(&ctl.acc_full[ab], (j >> 1) & 1, abort))) break;
      cfence_after();
      const int t = (int)blockIdx.x + j * (int)gridDim.x;
      const int c = t / nib, ib = t - c * nib;
      const int r = warp * 32 + lane, b = ib * 16 + (r >> 3);
      const int2 pq = __ldg(cls_pq + c);
      // this lane's output row (item b, member r % 8); rows of items past B are not stored
      const long long row_off = b < B ? (long long)b * y_stride + (long long)cmember(pq.x, pq.y, r & 7, M) * Z : -1;
      float2* ob = obuf + warp * 32 * 33;
      const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ab * S::kAcc);
#pragma unroll 1
      for (int z0 = 0; z0 < Z; z0 += 32) {
        uint32_t re[32], im[32];
        ctmem_ld32(tb + z0, re);
        ctmem_ld32(tb + Z + z0, im);
        // transpose through shared memory (rows padded to 33): then each of the warp's 32 rows is
        // written as 256 contiguous bytes
#pragma unroll
        for (int i = 0; i < 32; ++i) ob[lane * 33 + i] = make_float2(__uint_as_float(re[i]), __uint_as_float(im[i]));
        __syncwarp();
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
          const long long off = __shfl_sync(0xffffffffu, row_off, rr);
          if (off >= 0) Y[off + z0 + lane] = ob[rr * 33 + lane];
        }
        __syncwarp();
      }
      cfence_before();
      __syncwarp();
      if (lane == 0) cbar_arrive(&ctl.acc_empty[ab]);
    }
  } else if (warp < kCMmaWarp) {
    // ---------------------------------------------------------------- producers
    // task of a block: A row ra, frequencies 4 ha .. 4 ha + 3 of the block; B row z = ra (z < Z), the
    // same frequencies.  Each 8 lanes take 8 consecutive rows of one half (ra = 8 (pt / 16) + pt % 8,
    // ha = (pt / 8) % 2), so their 16-byte chunk stores meet 8 different bank groups of the swizzle.
    const int pt = (warp - kCEpiWarps) * 32 + lane;
    const int ra = ((pt >> 4) << 3) | (pt & 7), ha = (pt >> 3) & 1;
    const bool has_b = pt < 2 * Z;
    struct Regs {
      float4 a0, a1;  // U[f0 + 4 ha .. + 3] of row ra (two complex values each)
      float2 g[4];    // G[f0 + 4 hb + i][z]
    };
    auto load = [&](Regs& v, int it) {
      if (it >= my_iters) return;
      const int j = it / nkb, kb = it - j * nkb;
      const int t = (int)blockIdx.x + j * (int)gridDim.x;
      const int c = t / nib, ib = t - c * nib;
      const int f0 = kb * 8;
      const int b = ib * 16 + (ra >> 3);
      if (b < B) {
        const int2 pq = __ldg(cls_pq + c);
        const float4* src = reinterpret_cast<const float4*>(U + (size_t)b * u_stride +
                                                            (size_t)cmember(pq.x, pq.y, ra & 7, M) * F + f0 + 4 * ha);
        v.a0 = __ldg(src);
        v.a1 = __ldg(src + 1);
      } else {
        v.a0 = v.a1 = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (has_b) {
        const float2* g = Gc + ((size_t)c * F + f0 + 4 * ha) * Z + ra;
#pragma unroll
        for (int i = 0; i < 4; ++i) v.g[i] = __ldg(g + (size_t)i * Z);
      }
    };
    // 16-byte chunk ch of row r of a 64-byte-swizzled tile
    auto chunk = [](unsigned char* tile, int r, int ch) {
      return reinterpret_cast<uint4*>(tile + r * 64 + ((ch ^ ((r >> 1) & 3)) << 4));
    };
    auto stage = [&](const Regs& v, int it) -> bool {
      const int st = it % NS, ph = (it / NS) & 1;
      if (!__all_sync(0xffffffffu, cbar_wait(&ctl.empty[st], ph ^ 1, abort))) return false;
      uint4 h, l;
      // A row ra: Re U of frequencies 4 ha .. 4 ha + 3 at chunk ha, Im U at chunk 2 + ha
      split4(v.a0.x, v.a0.z, v.a1.x, v.a1.z, h, l);
      *chunk(a_hi(st), ra, ha) = h;
      *chunk(a_lo(st), ra, ha) = l;
      split4(v.a0.y, v.a0.w, v.a1.y, v.a1.w, h, l);
      *chunk(a_hi(st), ra, 2 + ha) = h;
      *chunk(a_lo(st), ra, 2 + ha) = l;
      if (has_b) {  // rows z (Re Y) and Z + z (Im Y)
        const int z = ra;
        split4(v.g[0].x, v.g[1].x, v.g[2].x, v.g[3].x, h, l);  // Re G
        *chunk(b_hi(st), z, ha) = h;
        *chunk(b_lo(st), z, ha) = l;
        *chunk(b_hi(st), Z + z, 2 + ha) = h;
        *chunk(b_lo(st), Z + z, 2 + ha) = l;
        split4(v.g[0].y, v.g[1].y, v.g[2].y, v.g[3].y, h, l);  // Im G
        *chunk(b_hi(st), Z + z, ha) = h;
        *chunk(b_lo(st), Z + z, ha) = l;
        h = make_uint4(h.x ^ 0x80000000u, h.y ^ 0x80000000u, h.z ^ 0x80000000u, h.w ^ 0x80000000u);  // -Im G
        l = make_uint4(l.x ^ 0x80000000u, l.y ^ 0x80000000u, l.z ^ 0x80000000u, l.w ^ 0x80000000u);
        *chunk(b_hi(st), z, 2 + ha) = h;
        *chunk(b_lo(st), z, 2 + ha) = l;
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) cbar_arrive(&ctl.full[st]);
      return true;
    };
    Regs v[kCAhead];
#pragma unroll
    for (int i = 0; i < kCAhead; ++i) load(v[i], i);
    for (int it = 0; it < my_iters; it += kCAhead) {
      bool ok = true;
#pragma unroll
      for (int i = 0; i < kCAhead; ++i) {
        if (it + i >= my_iters) break;
        if (!stage(v[i], it + i)) {
          ok = false;
          break;
        }
        load(v[i], it + i + kCAhead);
      }
      if (!ok) break;
    }
  } else {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(kCM, N2);
      int it = 0;
      bool ok = true;
      for (int j = 0; j < my_tiles && ok; ++j) {
        const int ab = j & 1;
        if (!cbar_wait(&ctl.acc_empty[ab], ((j >> 1) & 1) ^ 1, abort)) break;
        cfence_after();
        const uint32_t d = tmem + (uint32_t)(ab * S::kAcc);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int st = it % NS, ph = (it / NS) & 1;
          if (!cbar_wait(&ctl.full[st], ph, abort)) {
            ok = false;
            break;
          }
          cfence_after();
          const uint64_t dah = csw64_desc(csa(a_hi(st))), dal = csw64_desc(csa(a_lo(st)));
          const uint64_t dbh = csw64_desc(csa(b_hi(st))), dbl = csw64_desc(csa(b_lo(st)));
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {  // 8 tf32 = 32 bytes along K per instruction
            const uint64_t adv = (uint64_t)(2 * kk);
            umma_tf32(d, dah + adv, dbh + adv, idesc, (kb | kk) != 0);
            umma_tf32(d, dah + adv, dbl + adv, idesc, 1u);
            umma_tf32(d, dal + adv, dbh + adv, idesc, 1u);
          }
          cumma_commit(&ctl.empty[st]);
        }
        if (ok) cumma_commit(&ctl.acc_full[ab]);
      }
      // every MMA issued has completed before the CTA tears down
      cumma_commit(&ctl.drain);
      for (long long i = 0; i < kCSpin; ++i)
        if (cbar_try(&ctl.drain, 0)) break;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && ctl.abort) atomicOr(status, 2);
  if (warp == 0) {
    cfence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * S::kAcc)
                 : "memory");
  }
}

template <int N2>
cudaError_t launch_cu(const float2* U, long long u_stride, const float2* Gc, const int2* cls_pq, int ncls, int M,
                      int F, float2* Y, long long y_stride, int B, int* status, cudaStream_t s) {
  using S = CShape<N2>;
  static bool configured = false;
  static int sms = 0;
  if (!configured) {
    const cudaError_t e =
        cudaFuncSetAttribute(contract_umma_kernel<N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    configured = true;
  }
  const long long ntiles = (long long)ncls * ((B + 15) / 16);
  const int grid = (int)std::min<long long>(ntiles, sms);
  contract_umma_kernel<N2><<<grid, kCThreads, S::kSmem, s>>>(U, u_stride, Gc, cls_pq, ncls, M, F, Y, y_stride, B,
                                                             status);
  return cudaGetLastError();
}

}  // namespace

bool contract_umma_supported(int M, int F, int Z, int B, long long u_stride, long long y_stride) {
  return M >= 2 && (M & (M - 1)) == 0 && F >= 8 && F % 8 == 0 && (Z == 32 || Z == 64 || Z == 128) &&
         B >= 1 && u_stride % 2 == 0 && y_stride % 2 == 0;
}

cudaError_t launch_contract_umma(const float2* U, long long u_stride, const float2* Gc, const int2* cls_pq, int ncls,
                                 int M, int F, int Z, float2* Y, long long y_stride, int B, int* status,
                                 cudaStream_t s) {
  if (!contract_umma_supported(M, F, Z, B, u_stride, y_stride) || !status || ncls < 1 ||
      reinterpret_cast<uintptr_t>(U) % 16 != 0 || reinterpret_cast<uintptr_t>(Y) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(Gc) % 8 != 0)
    return cudaErrorInvalidValue;
  switch (Z) {
    case 32: return launch_cu<64>(U, u_stride, Gc, cls_pq, ncls, M, F, Y, y_stride, B, status, s);
    case 64: return launch_cu<128>(U, u_stride, Gc, cls_pq, ncls, M, F, Y, y_stride, B, status, s);
    default: return launch_cu<256>(U, u_stride, Gc, cls_pq, ncls, M, F, Y, y_stride, B, status, s);
  }
}

}  // namespace nursd
