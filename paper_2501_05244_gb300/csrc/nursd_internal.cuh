// Internal declarations of libnursd (not part of the public C ABI).
//
// Data layouts (all row-major, the last index contiguous):
//   phasors      P    [L][F]            complex64, f fastest
//   fine grid    Bf   [W][W][F]         the non-zero window of the oversampled
//                                       NUFFT grid (fine index g = i + g0)
//   row spectra  R1   [W][M][F]         after the FFT along x, kx in I_M
//   spectrum     U    [M][M][F]         (ky, kx) in I_M^2, f fastest
//   transfer fn  Gc   [ncls][F][Z]      one entry per 8-fold symmetry class
//   depth spectra Y   [M][M][Z]         sum over f of U * Ghat
//   half IDFT    T1   [M][N][Z]         after the inverse FFT along kx
//   volume       V    [Z][N][N]         complex64 or magnitude float32
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/nursd.h"

namespace nursd {

// Programmatic dependent launch: a kernel launched by launch_pdl may start, and run the part of its
// prologue that touches no global memory written by others, while the previous kernel in the stream
// finishes.  Such a kernel calls pdl_wait() before its first read of what that kernel wrote and
// before its first global write; pdl_wait() returns once the previous kernel has completed and its
// writes are visible (at once when there is no programmatic dependency).  pdl_trigger() lets the next
// kernel launch early once every CTA of this grid has called it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Checks of data-dependent indices, compiled in with -DNURSD_CHECKED (the library's checked build):
// a failed check sets status bit 16 (NURSD_ERR_CUDA from nursd_sync_status) and the access is
// skipped; without the flag a check is the constant true.
#ifdef NURSD_CHECKED
#define NURSD_CHECK(cond, status) ((cond) ? true : (((status) ? atomicOr((status), 16) : 0), false))
#else
#define NURSD_CHECK(cond, status) true
#endif

constexpr int kTile = 16;          // spreading tile edge (fine cells)
constexpr int kTwiddleLog = 12;    // shared FFT twiddle table has 2^12 entries, then the per-thread rows below
constexpr int kMaxKernelWidth = 8;
constexpr int kMaxBatch = 256;     // reconstructions per batched call

// The FFT table (kTwiddleEntries complex64 values):
//   [0, 2^12)                   e^{-2 pi i q / 2^12}
//   kTw2Offset + 16 k + t       W_256^{k t}            (k, t < 16; the radix-16 x 16 middle stage)
//   tw3_offset(lg) + R j + t    W_{2^lg}^{j t}         (j < 256, t < R = 2^lg / 256; the last stage)
//   tw32_offset(lg) + R j + t   W_{2^lg}^{j t}         (j < 32, t < R = 2^lg / 32; the second stage of
//                                                       the radix-32 form, lg = 9, 10, then 8)
// so that a thread reads its whole row of twiddles at one base address.
constexpr int kTw2Offset = 1 << kTwiddleLog;
constexpr int kTw3Offset = kTw2Offset + 256;
__host__ __device__ constexpr int tw3_offset(int lg) { return kTw3Offset + (lg == 9 ? 0 : (lg == 10 ? 512 : 1536)); }
constexpr int kTw32Offset = kTw3Offset + 512 + 1024 + 2048;
__host__ __device__ constexpr int tw32_offset(int lg) { return kTw32Offset + (lg == 9 ? 0 : (lg == 10 ? 512 : 1536)); }
constexpr int kTwiddleEntries = kTw32Offset + 512 + 1024 + 256;
// Entry e of the table is exp(-2 pi i num / 2^lg).
__host__ __device__ inline void twiddle_exponent(int e, int* num, int* lg) {
  if (e < kTw2Offset) {
    *num = e;
    *lg = kTwiddleLog;
  } else if (e < kTw3Offset) {
    const int r = e - kTw2Offset;
    *num = (r >> 4) * (r & 15);
    *lg = 8;
  } else if (e < kTw32Offset) {
    const int l = e < tw3_offset(10) ? 9 : (e < tw3_offset(11) ? 10 : 11);
    const int r = e - tw3_offset(l), R = 1 << (l - 8);
    *num = (r / R) * (r % R);
    *lg = l;
  } else {
    const int l = e < tw32_offset(10) ? 9 : (e < tw32_offset(8) ? 10 : 8);
    const int r = e - tw32_offset(l), R = 1 << (l - 5);
    *num = (r / R) * (r % R);
    *lg = l;
  }
}

__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// ---------------------------------------------------------------- panel FFT
// One CTA transforms CHI*CLO "channels" of one batch item along the FFT axis.
// Input element (b, i, hi, lo) sits at in[b*in_sb + i*in_si + hi*in_shi + lo*in_slo]
// and lands at FFT position (i + in_off) mod n; output o is FFT bin
// (o + out_off) mod n and goes to out[b*out_sb + o*out_si + hi*out_shi + lo*out_slo].
struct PanelArgs {
  const float2* in;
  float2* out;
  float* out_mag;  // if non-null: write |value| here instead of out
  long long in_sb, in_si, in_shi, in_slo;
  long long out_sb, out_si, out_shi, out_slo;
  int nin, in_off;
  int nout, out_off;
  int hi_total, lo_total;  // channel extents
  int CHI, CLO;            // panel shape, CHI*CLO == CP
  int batch;
  const float* mul_i;  // optional real factor per input index (applied on load)
  const float* mul_o;  // optional real factor per output index
  const float* mul_b;  // optional real factor per batch item
  float scale;
  int load_i_fastest;    // consecutive threads load consecutive i (FFT axis contiguous in memory)
  int store_hi_fastest;  // consecutive threads store consecutive hi channels
  int store_o_fastest;   // consecutive threads store consecutive outputs o
  const float2* twiddle;  // the FFT table (kTwiddleEntries values, 16-byte aligned)
  // Transfer products formed while the window is staged (radix-32 kernels, CP = 8): with
  // prod_g set, channel 4 j + zz of panel chunk c (f0 = 2 c, j < 2, zz < 4) at window row i of
  // batch item b is in[b in_sb + i in_si + f0 + j] * prod_g[class(i - nin/2, b - nin/2)][f0 + j]
  // [prod_z0 + zz], the table [class][prod_F][prod_Z] of the symmetry classes
  // {(+-p, +-q), (+-q, +-p)} at index p (p + 1) / 2 + q.
  const float2* prod_g;
  int prod_F, prod_Z, prod_z0;
};

// Launches the panel FFT of length 2^logn (4 <= 2^logn <= 2048). Returns a cudaError_t.
cudaError_t launch_panel_fft(int logn, bool inverse, const PanelArgs& a, cudaStream_t s);
// Length 256 in the persistent radix-32 register form (16-channel panels); cudaErrorNotSupported
// (nothing launched) when the pass has too few panels for it.
cudaError_t launch_panel_fft32_256(bool inverse, const PanelArgs& a, cudaStream_t s);
// Panel width (channels per CTA) used for a given transform length.
int panel_width(int logn);
// Register-resident kernels for 2^9..2^11 (fft_reg.cu).
int panel_width_reg(int logn);
cudaError_t launch_panel_fft_reg(int logn, bool inverse, const PanelArgs& a, cudaStream_t s);
cudaError_t launch_panel_bluestein_reg(int logn, const PanelArgs& a, const float2* cpre, const float2* bhat,
                                       const float2* cpost, cudaStream_t s);
// Bluestein scaled DFT along the panel axis: window * cpre[i] -> FFT_n -> * bhat[bin] ->
// inverse FFT_n -> kept bins * cpost[o] (store order: channels fastest).
cudaError_t launch_panel_bluestein(int logn, const PanelArgs& a, const float2* cpre, const float2* bhat,
                                   const float2* cpost, cudaStream_t s);

// ------------------------------------------------------------- temporal DFT
// P[l][f] = w_f sum_n h[l][n] * B[n][2f..2f+1] as a real GEMM C[L][2F] = H[L][T] B[T][2F] diag(wcol)
// on the tensor cores; Bh/Bl are the fp16 head and tail of the unit-modulus B^T, [2F][T] (__half),
// wcol [2F] the weight of each column (w_f twice).  row_slot (optional): row l of C is written at
// row row_slot[l] (the spread's sorted order).
//
// Range: every operand is split into an fp16 head and tail, which carries ~22 bits of a value
// whose row max m lies in [2^-3, 65504).  Rows outside that window are listed in a TemporalFix
// (row, exponent e with m 2^-e in [2^14, 2^15), batch item) by the first launch, and a gather
// launch recomputes exactly those rows from h 2^-e, scaling the result by 2^e.
constexpr int kRowInRange = 0x7fffffff;
__device__ __forceinline__ int temporal_row_exponent(float m) {
  if (m == 0.f || !isfinite(m) || (m >= 0.125f && m < 65504.f)) return kRowInRange;
  return ilogbf(m) - 14;
}
struct TemporalFix {
  int* count;  // device: rows listed; zero between calls (the gather launch clears it)
  int* done;   // device: gather CTAs that have read count (zero between calls)
  int4* list;  // device [cap]: {row, e, batch item, 0}
  int cap;
};
// Gather launch prologue, thread 0 of each CTA: reads the listed-row count, and the last CTA to do
// so clears count and done for the next call.  Returns the count.
__device__ __forceinline__ int temporal_fix_take(const TemporalFix& fix) {
  const int n = *(volatile int*)fix.count;
  __threadfence();
  if (atomicAdd(fix.done, 1) == (int)(gridDim.x * gridDim.y * gridDim.z) - 1) {
    __threadfence();
    *(volatile int*)fix.count = 0;
    *(volatile int*)fix.done = 0;
  }
  return n;
}
cudaError_t launch_temporal_tc(const float* h, const void* Bh, const void* Bl, const float* wcol, float* C, int L,
                               int T, int twoF, const TemporalFix& fix, cudaStream_t s,
                               const int* row_slot = nullptr);

// The same transform with tcgen05.mma (temporal_umma.cu), for T % 32 == 0 and 2F in {32, 64, 128, 256}.
// TMA descriptors of B's head and tail ([2F][T] fp16) are encoded once per plan.
struct TemporalMaps {
  CUtensorMap hi;
  CUtensorMap lo;
  int ok;
};
bool temporal_umma_supported(int T, int twoF);
bool make_temporal_maps(const void* Bh, const void* Bl, int T, int twoF, TemporalMaps* m);
// status: bit 4 is set if a barrier wait timed out (the output is then incomplete).  Both the
// first launch and the gather launch of listed rows (see TemporalFix) are issued on s.
cudaError_t launch_temporal_umma(const TemporalMaps& m, const float* h, const float* wcol, float* C, int L, int T,
                                 int twoF, const TemporalFix& fix, int* status, cudaStream_t s,
                                 const int* row_slot = nullptr);

// Ragged batch of temporal transforms: item b has L[b] rows at A[b] -> C[b];
// tile_start[b] = number of 128 x 128 output tiles of items 0..b-1.
struct TemporalBatch {
  int n;
  const float* A[kMaxBatch];
  float* C[kMaxBatch];
  int L[kMaxBatch];
  int tile_start[kMaxBatch + 1];
};
cudaError_t launch_temporal_tc_batched(const TemporalBatch& bt, const void* Bh, const void* Bl, const float* wcol,
                                       int T, int twoF, const TemporalFix& fix, int* counter, cudaStream_t s);
// The listed rows of every item of bt (TemporalFix entries {row, e, item, 0}) recomputed from h 2^-e
// by the mma.sync form (the second launch of the batched transforms).
cudaError_t launch_temporal_tc_gather(const TemporalBatch& bt, const void* Bh, const void* Bl, const float* wcol,
                                      int T, int twoF, const TemporalFix& fix, cudaStream_t s);
// The tcgen05 transform of every item of bt in one persistent launch (bt.tile_start counting 128-row
// tiles); rows outside the split's window are listed in fix for launch_temporal_tc_gather.
cudaError_t launch_temporal_umma_batched(const TemporalMaps& m, const TemporalBatch& bt, const float* wcol, int T,
                                         int twoF, const TemporalFix& fix, int* status, cudaStream_t s);

// ---------------------------------------------------------------- points
struct PointsArgs {
  const float* xy;     // [L][2] metres
  int L;
  double cx, cy, inv_fine_pitch;  // fine coordinate u = (x - c) * inv_fine_pitch
  double half_extent;             // |x - c| <= half_extent is in range
  int g0;                         // fine index of window cell 0
  int W, tiles;                   // window width and tiles per axis
  int width;                      // ES kernel width w
  float beta;                     // ES kernel shape
  int* status;                    // device error word
};
// Prepare and sort the relay samples by bin = (tile column, edge flag, footprint row),
// nbins = points_bins(W, tiles).  Scratch in original order: bin_of [L],
// i0_orig [L], w_orig [L][2w]; counts needs 2*nbins ints.  Sorted outputs:
// sorted_l [L] (original index), i0_sorted, w_sorted, and bin_start [nbins+1].
int points_bins(int W, int tiles);
// frac_sorted (optional) receives u - i0 per axis of each sorted sample; slot_of (optional) the
// inverse of sorted_l (the sorted slot of each sample).
cudaError_t launch_points(const PointsArgs& a, int* bin_of, int2* i0_orig, float* w_orig, int* counts,
                          int* bin_start, int* sorted_l, int2* i0_sorted, float* w_sorted, cudaStream_t s,
                          float2* frac_orig = nullptr, float2* frac_sorted = nullptr, int* slot_of = nullptr);
// The same for the n items of a batched call (a.L and a.xy unused): item b has items.L[b] samples at
// items.xy[b]; its per-sample arrays (scratch and sorted) start at b * pts, its counts at b * 2 nbins
// and its bin_start at b * (nbins + 1).  An item with no samples gets an all-zero bin_start.
struct PointsItems {
  int L[kMaxBatch];
  const float* xy[kMaxBatch];
};
cudaError_t launch_points_batched(const PointsArgs& a, const PointsItems& items, int n, long long pts, int* bin_of,
                                  int2* i0_orig, float* w_orig, int* counts, int* bin_start, int* sorted_l,
                                  int2* i0_sorted, float* w_sorted, float2* frac_orig, float2* frac_sorted,
                                  int* slot_of, cudaStream_t s);

// ---------------------------------------------------------------- spread
// sorted_l == nullptr: P is already in sorted-slot order (row s of P is sorted sample s).  rows: tile
// height (spread_rows_supported: 4, 8 or 16; W must be a multiple of it).
bool spread_rows_supported(int rows);
// n items of a batched call (grid z): item b's phasors at P + b p_stride, its sorted per-sample arrays
// at b pts (weights b pts 2w), its bin_start at b bstride and its window at fine + b fine_stride.
struct SpreadItems {
  int n = 1;
  long long p_stride = 0, pts = 0, fine_stride = 0;
  int bstride = 0;
  int* status = nullptr;  // checked build: a staged sample whose first footprint row misses the tile's
                          // reach (a bin out of order) sets bit 16 and is not spread
  // 3D slices (item j = fine z cell gz_first + j): with uz (the samples' fine z coordinates, slot
  // order), samples whose z footprint misses the item's cell (zero phasors there) are skipped
  const float* uz = nullptr;
  int gz_first = 0;
};
cudaError_t launch_spread(const float2* P, int F, const int* bin_start, const int* sorted_l,
                          const int2* i0, const float* wts, int width, int tiles, int W,
                          float2* fine, cudaStream_t s, int rows = 8, const SpreadItems& items = SpreadItems());

// ------------------------------------------------------------- contraction
// Y[k][z] = sum_f U[k][f] * Gc[cls(k)][f][z] for every mode k of every class.
// status (device int, may be null): bulk-copy form's wait time-outs set bit 2.
cudaError_t launch_contract(const float2* U, const float2* Gc, const int2* cls_pq, int ncls, int M,
                            int F, int Z, float2* Y, cudaStream_t s, int* status = nullptr);

// Batched: B spectra U + b*u_stride -> Y + b*y_stride, consecutive CTAs sweeping the
// batch for one class group so that each table block is read from HBM once.
cudaError_t launch_contract_batched(const float2* U, long long u_stride, const float2* Gc, const int2* cls_pq,
                                   int ncls, int M, int F, int Z, float2* Y, long long y_stride, int B,
                                   cudaStream_t s, int* status = nullptr);
// Test only: the bound (mbarrier polls) of the bulk-copy contraction's data waits on the current device
// (polls < 0: the default; 0: give up at the first wait); a wait that runs out sets status bit 2, drains
// the warp's copies and returns.
cudaError_t set_contract_wait_limit(long long polls, cudaStream_t s);
// Adjoint: R[k][f] = sum_z Yt[k][z] * conj(GcT[cls(k)][z][f]).
cudaError_t launch_contract_adjoint(const float2* Yt, const float2* GcT, const int2* cls_pq, int ncls, int M, int F,
                                    int Z, float2* R, cudaStream_t s, int* status = nullptr);
// Tensor-core form with the table as the A operand (contract_tc.cu): for every mode k of every class,
// out[k][r] = sum_i A[cls(k)][r][i] X[k][i] (conj = false) or sum_i conj(A[cls(k)][r][i]) X[k][i]
// (conj = true), table [ncls][rows][inner].  The forward is (X = U, A = GcT, rows Z, inner F), the
// adjoint (X = Y, A = Gc, rows F, inner Z, conj).  Needs rows = 128 and inner a multiple of 16;
// cudaErrorInvalidValue otherwise.  status: wait time-outs set bit 2.
bool contract_tc_supported(int M, int rows, int inner);
cudaError_t launch_contract_tc(const float2* X, const float2* table, const int2* cls_pq, int ncls, int M, int rows,
                               int inner, bool conj, float2* out, cudaStream_t s, int* status);

// ------------------------------------------------------------ interpolation
// Type-2 interpolation at the sorted relay samples from a channel-last fine
// grid [W][W][F]: out[l][f] = scale * sum_taps fine[i0y+ty][i0x+tx][f] wx wy.
// With gxy: the same taps on fine_dx / fine_dy, the type-2 grids of kx R and
// ky R, give d/d(x, y) of that value as i dudx times their interpolants, reduced
// against P: gxy[l] = scale * dudx * Im sum_f P[l][f] conj(interpolant).
struct InterpArgs {
  const float2* fine;         // value grid (read when out is set)
  const float2* fine_dx;      // derivative grids (read when gxy is set)
  const float2* fine_dy;
  int W, F, width, L;
  float beta, dudx;           // ES shape; d theta / dx = 2 pi / (M delta)
  const int* sorted_l;
  const int2* i0;
  const float* wts;           // [L][2w] sorted
  float scale;
  float2* out;                // [L][F] (original sample order) or null
  const float2* P;            // [L][F] for the gradient reduction
  float* gxy;                 // [L][2] or null
};
cudaError_t launch_interp_points(const InterpArgs& a, cudaStream_t s);

// Type-2 interpolation at per-plane voxels from a plane-major fine grid
// [Z][W][W]: out[z][v] = scale * sum_taps fine[z][..][..] wx wy, positions
// vox[z][v] (metres) mapped like relay samples; out-of-aperture voxels flag
// status bit 1 and give 0.
struct PlaneInterpArgs {
  const float2* fine;
  int W, Z, K, width, g0;
  float beta;
  double cx, cy, inv_fine_pitch, half_extent;
  const double* plane_scale;  // [Z] or null: plane z's lattice pitch over the plan's (inv_fine_pitch
                              // divided by it, half_extent multiplied)
  const float* vox;  // [Z][K][2]
  float scale;
  float2* out;       // [Z][K]
  int* status;
};
cudaError_t launch_interp_planes(const PlaneInterpArgs& a, cudaStream_t s);

// ------------------------------------------------------- transfer function
// g[jy][jx][zb*F + f] = exp(i k_f r)/r, r = sqrt((jx d)^2 + (jy d)^2 + z_zb^2), FP64 phase;
// d = d_pitch[zb] when d_pitch is non-null (SRSD's scaled lattice), else `pitch`.
cudaError_t launch_gtf_generate(float2* g, int M, double pitch, const double* d_z, int ZB,
                                const double* d_k, int F, cudaStream_t s, const double* d_pitch = nullptr);
// Gs[((z0 + zb) * ncls + c) * F + f] = Gfull[rep(c)][zb*F + f] (per-depth blocks, f fastest)
cudaError_t launch_gtf_compress_depthmajor(const float2* Gfull, const int2* cls_pq, int ncls, int M, int F, int ZB,
                                           int z0, float2* Gs, cudaStream_t s);
// ------------------------------------------- batched contraction on the tensor cores (contract_umma.cu)
// Y[b][k][z] = sum_f U[b][k][f] * Gc[cls(k)][f][z] for every mode k and item b < B (item b's spectrum
// at U + b u_stride, its depth spectra at Y + b y_stride), as tcgen05 kind::tf32 products with a
// head/tail split (FP32 accuracy).  Supported for M a power of two, F a multiple of 8 and Z in
// {32, 64, 128}; status (device int) gets bit 2 when a bounded wait gave up.
bool contract_umma_supported(int M, int F, int Z, int B, long long u_stride, long long y_stride);
cudaError_t launch_contract_umma(const float2* U, long long u_stride, const float2* Gc, const int2* cls_pq, int ncls,
                                 int M, int F, int Z, float2* Y, long long y_stride, int B, int* status,
                                 cudaStream_t s);
// ------------------------------------------------- SRSD by interpolation (srsd_interp.cu)
// Yh [L][L][F] at index m + L/2 (periodic in m).
// Both taps and the contraction in one pass for every depth z in zlist[0 .. nz) (device list; 4 <= w <= 8;
// the tap table of each depth must advance by 0, 1 or 2 cells per mode index):
// Y[k][z] = sum_f Gs[z][class(k)][f] sum_ty wt[z][ky][ty] sum_tx wt[z][kx][tx] Yh[m0[z][ky] + ty][m0[z][kx] + tx][f].
// When srsd_interp_adds(F, L, w) the channels of a mode are summed into Y, whose listed depths must then
// be zero on entry.  status (device int): bit 2 when a bounded barrier wait gave up, bit 8 when a tap
// table breaks the step rule (nothing is written for the modes concerned).
bool srsd_interp_adds(int F, int L, int w);
cudaError_t launch_srsd_interp_xy_contract(const float2* Yh, int L, int M, int F, int Z, const int* zlist, int nz,
                                           int w, const int* m0, const float* wt, const float2* Gs, int ncls,
                                           float2* Y, int* status, cudaStream_t s);
// ------------------------------------------------ 3D NURSD (nursd3d.cu)
// uz_sorted[s] = h[sorted_l[s]] inv_fine_dz (|h| > half_extent: status bit 1, no weight).
cudaError_t launch_z_coords(const float* h, const int* sorted_l, int L, double inv_fine_dz, double half_extent,
                            float* uz_sorted, int* status, cudaStream_t s);
// Pz[j][s][f] = P[sorted_l[s]][f] phi(2 (gz - uz[s]) / w), gz = gz_first + j for j < n (slot order;
// slice j at Pz + j pz_stride).
cudaError_t launch_z_slice_phasors(const float2* P, const int* sorted_l, const float* uz, int L, int F, int gz_first,
                                   int n, long long pz_stride, int w, float beta, float2* Pz, cudaStream_t s);
// What[k][f] = scale sum_kz U3[k][kz][f] G3[k][kz][f] for nk lateral modes k.
cudaError_t launch_kz_sum(const float2* U3, const float2* G3, long long nk, int Mz, int F, float scale, float2* What,
                          cudaStream_t s);
// ------------------------------------------------ subsampled acquisition (resample.cu)
// kept [Nc][Nc][F] = full[::D, ::D]; full [N][N][F] from kept by nearest (linear = 0) or linear interpolation.
cudaError_t launch_subsample(const float2* full, float2* kept, int N, int F, int D, cudaStream_t s);
cudaError_t launch_upsample(const float2* kept, float2* full, int N, int F, int D, int linear, cudaStream_t s);
// ---------------------------------------------------------- per-frequency forms (illum.cu)
// Y[k][zz*F + f] = U[k][f] * Gc[class(k)][f][z0 + zz] for zz < zg (no sum over f), U and Y
// mode-major [M][M][...] with mode (kx, ky) at (ky + M/2) M + (kx + M/2).
cudaError_t launch_transfer_depths(const float2* U, const float2* Gc, int M, int F, int Z, int z0, int zg, float2* Y,
                                   cudaStream_t s);
struct IllumArgs {
  double xp, yp, zp;     // illumination point (m), relay frame
  double cx, cy, pitch;  // voxel (mx, my) of a plane at (cx + (mx - N/2) pitch, cy + (my - N/2) pitch)
  const double* depth;   // device [Z] plane depths (m)
  const double* kap;     // device [F] k_f / (2 pi) = w_f / (2 pi c), cycles per metre
  double dkap;           // kap[f + 1] - kap[f] when equispaced
  int equispaced;        // kap[f] = kap[0] + f dkap to FP64 rounding
};
// out[z0 + zz][my][mx] = sum_f exp(+i k_f |x_p - x_v|) V[zz*cz + f*cf][my][mx], V channel-major
// [zg*F][N][N] (channel of depth zz and frequency f at zz*cz + f*cf), out [Z][N][N].
cudaError_t launch_illum_sum(const float2* V, int F, int N, int z0, int zg, int cz, int cf, const IllumArgs& a,
                             float2* out, cudaStream_t s);
// The same with V channel-last [N][N][zg*F], the channel of depth zz and frequency f at f*zg + zz.
cudaError_t launch_illum_sum_cl(const float2* V, int F, int N, int z0, int zg, const IllumArgs& a, float2* out,
                                cudaStream_t s);
// out[t][z0 + zz][my][mx] = sum_f A[t][f] V[zz*cz + f*cf][my][mx], A [T][F], out [T][Z][N][N].
cudaError_t launch_frames_sum(const float2* V, int F, int N, int Z, int z0, int zg, int cz, int cf, const float2* A,
                              int T, float2* out, cudaStream_t s);
// SRSD contraction for one depth: Y[k][z] = sum_f Phat[k][f] * Gs_z[cls(k)][f].
cudaError_t launch_contract_depth(const float2* Phat, const float2* Gs_z, const int2* cls_pq, int ncls, int M, int F,
                                  int Z, int z, float2* Y, cudaStream_t s);
// Gc[(c*F + f)*Z + z0 + zb] = Gfull[rep(c)][zb*F + f]; with GcT non-null also
// GcT[(c*Z + z0 + zb)*F + f] = the same value.
cudaError_t launch_gtf_compress(const float2* Gfull, const int2* cls_pq, int ncls, int M, int F,
                                int ZB, int Z, int z0, float2* Gc, float2* GcT, cudaStream_t s);

}  // namespace nursd
