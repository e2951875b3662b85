// NUFFT type 1 that allocates no device memory.
//
// The plan-based path (nursd_plan_create + nursd_set_points + nursd_nufft1)
// obtains its workspace with cudaMalloc.  Some callers cannot do that: engines
// that own every byte of device memory through a pre-reserved pool, or plugins
// running inside such an engine, where an extra cudaMalloc is forbidden (it can
// synchronise the device and it escapes the pool's accounting).  This file gives
// them one entry point that runs the same kernels -- relay-sample preparation
// and sort, spread, the two FFT passes with deconvolution -- with all of its
// scratch in a fixed, file-scope device array.
//
// The array (kNoAllocScratchBytes) is part of the library image: every GPU that
// loads libnursd holds it until the process exits.  Its device address is looked
// up once per device with cudaGetSymbolAddress; host code never passes the
// symbol itself to a kernel.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "nursd_internal.cuh"

using namespace nursd;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(24) << 20;  // 24 MiB, shared by every call
constexpr size_t kTableBytes = size_t(128) << 10;         // FFT table + quadrature nodes
constexpr int kQuadNodes = 256;
static_assert(sizeof(float2) * kTwiddleEntries + 2 * sizeof(double) * kQuadNodes <= kTableBytes,
              "fixed tables exceed their part of the scratch array");
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_nursd_noalloc_scratch[kNoAllocScratchBytes];

struct DeviceScratch {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_nursd_noalloc_scratch on this device
  CUcontext ctx = nullptr;        // the context that address and the tables belong to
};
std::mutex g_mutex;
DeviceScratch g_devices[kMaxDevices];

// Fixed tables (once per device): the FFT table (twiddle_exponent) and
// 256-node Gauss-Legendre nodes/weights on [-1, 1] (Newton's method on P_n).
__global__ void noalloc_tables_kernel(float2* twiddle, double* gx, double* gw) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kTwiddleEntries) {
    int num = 0, lg = 0;
    twiddle_exponent(t, &num, &lg);
    double s, c;
    sincospi(-2.0 * num / (double)(1 << lg), &s, &c);
    twiddle[t] = make_float2((float)c, (float)s);
  }
  if (t < kQuadNodes) {
    const int n = kQuadNodes;
    double z = cospi((t + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 1; j < n; ++j) {
        const double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    gx[t] = z;
    gw[t] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// 1 / psi_hat(k) for k in I_M: psi_hat(k) = (w/2) int_{-1}^{1} phi(z) cos(pi k w z / nf) dz.
__global__ void noalloc_deconv_kernel(const double* gx, const double* gw, int M, int nf, int w, double beta,
                                      float* dec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double k = i - M / 2;
  double s = 0.0;
  for (int j = 0; j < kQuadNodes; ++j) {
    const double z = gx[j];
    const double phi = fabs(z) < 1.0 ? exp(beta * (sqrt(1.0 - z * z) - 1.0)) : 0.0;
    s += gw[j] * phi * cospi(k * w * z / nf);
  }
  dec[i] = (float)(1.0 / (0.5 * w * s));
}

int from_cuda(cudaError_t e) { return e == cudaSuccess ? NURSD_OK : NURSD_ERR_CUDA; }

// Lays out 256-byte-aligned regions of the per-call part of the scratch array.
struct Layout {
  size_t used = 0;
  template <class T>
  size_t take(size_t count) {
    const size_t off = (used + 255) & ~size_t(255);
    used = off + sizeof(T) * (count ? count : 1);
    return off;
  }
};

// The current context, through the driver entry point (the library does not link the driver).
CUcontext current_context() {
  using Fn = CUresult (*)(CUcontext*);
  static Fn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<Fn>(p);
    else
      cudaGetLastError();
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Once per device and context, with that device current: look up the array's device address and fill
// the fixed tables (synchronising `s`).  A new context on the device (after cudaDeviceReset, say) has
// its own copy of the array, so the address and tables are taken again.
int device_scratch(cudaStream_t s, unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NURSD_ERR_CUDA;
  if (cudaFree(nullptr) != cudaSuccess) return NURSD_ERR_CUDA;  // make sure the device's context exists
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceScratch& d = g_devices[dev];
  if (!d.ready || d.ctx != ctx) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_nursd_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      return NURSD_ERR_CUDA;
    }
    unsigned char* base = static_cast<unsigned char*>(ptr);
    float2* tw = reinterpret_cast<float2*>(base);
    double* gx = reinterpret_cast<double*>(base + sizeof(float2) * kTwiddleEntries);
    double* gw = gx + kQuadNodes;
    noalloc_tables_kernel<<<(kTwiddleEntries + 255) / 256, 256, 0, s>>>(tw, gx, gw);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return NURSD_ERR_CUDA;
    d.base = base;
    d.ctx = ctx;
    d.ready = true;
  }
  *out = d.base;
  return NURSD_OK;
}

}  // namespace

extern "C" int nursd_nufft1_noalloc(int32_t N, double pitch, double center_x, double center_y, int32_t kernel_width,
                                    int32_t L, const float* d_xy, int32_t F, const nursd_c64* d_phasor,
                                    nursd_c64* d_spectrum, nursd_stream_t stream) {
  if (N < 8 || N > 512 || (N & (N - 1)) != 0) return NURSD_ERR_UNSUPPORTED;
  if (!(pitch > 0) || !std::isfinite(pitch) || !std::isfinite(center_x) || !std::isfinite(center_y))
    return NURSD_ERR_INVALID_ARG;
  if (kernel_width < 4 || kernel_width > kMaxKernelWidth) return NURSD_ERR_UNSUPPORTED;
  if (L < 0 || F < 1 || F > 256 || !d_spectrum) return NURSD_ERR_INVALID_ARG;
  if (L > 0 && (!d_xy || !d_phasor)) return NURSD_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_xy) | reinterpret_cast<uintptr_t>(d_phasor) |
       reinterpret_cast<uintptr_t>(d_spectrum)) % 8 != 0)
    return NURSD_ERR_INVALID_ARG;

  // geometry, exactly as a plan derives it
  const int M = 2 * N, nf = 2 * M, w = kernel_width;
  const int W = (2 * N + w + 2 + kTile - 1) / kTile * kTile;
  const int tiles = W / kTile, g0 = -W / 2, nbins = points_bins(W, tiles);
  const float beta = (float)(2.30 * w);

  // regions of the per-call part; reject sizes that do not fit before touching the device
  Layout lay;
  const size_t o_dec = lay.take<float>(M), o_status = lay.take<int>(1), o_bin = lay.take<int>(L),
               o_i0o = lay.take<int2>(L), o_wo = lay.take<float>((size_t)L * 2 * w),
               o_cnt = lay.take<int>((size_t)2 * nbins), o_bs = lay.take<int>(nbins + 1),
               o_sl = lay.take<int>(L), o_i0s = lay.take<int2>(L), o_ws = lay.take<float>((size_t)L * 2 * w),
               o_fine = lay.take<float2>((size_t)W * W * F), o_r1 = lay.take<float2>((size_t)W * M * F);
  if (lay.used > kNoAllocScratchBytes - kTableBytes) return NURSD_ERR_UNSUPPORTED;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  int rc = device_scratch(s, &base);
  if (rc != NURSD_OK) return rc;
  const float2* tw = reinterpret_cast<const float2*>(base);
  const double* gx = reinterpret_cast<const double*>(base + sizeof(float2) * kTwiddleEntries);
  const double* gw = gx + kQuadNodes;
  unsigned char* call = base + kTableBytes;
  float* dec = reinterpret_cast<float*>(call + o_dec);
  int* status = reinterpret_cast<int*>(call + o_status);
  int* bin_of = reinterpret_cast<int*>(call + o_bin);
  int2* i0_orig = reinterpret_cast<int2*>(call + o_i0o);
  float* w_orig = reinterpret_cast<float*>(call + o_wo);
  int* counts = reinterpret_cast<int*>(call + o_cnt);
  int* bin_start = reinterpret_cast<int*>(call + o_bs);
  int* sorted_l = reinterpret_cast<int*>(call + o_sl);
  int2* i0_sorted = reinterpret_cast<int2*>(call + o_i0s);
  float* w_sorted = reinterpret_cast<float*>(call + o_ws);
  float2* fine = reinterpret_cast<float2*>(call + o_fine);
  float2* R1 = reinterpret_cast<float2*>(call + o_r1);

  // The array keeps the previous call's contents.  Everything below is fully rewritten before it is
  // read (the sort writes every count and bin start, the spread writes every window cell).  The status
  // word only absorbs the sort's out-of-aperture flags, which this entry point does not report.
  noalloc_deconv_kernel<<<(M + 127) / 128, 128, 0, s>>>(gx, gw, M, nf, w, (double)beta, dec);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    PointsArgs a;
    a.xy = d_xy;
    a.L = L;
    a.cx = center_x;
    a.cy = center_y;
    a.inv_fine_pitch = 2.0 / pitch;
    a.half_extent = 0.5 * N * pitch;
    a.g0 = g0;
    a.W = W;
    a.tiles = tiles;
    a.width = w;
    a.beta = beta;
    a.status = status;
    e = launch_points(a, bin_of, i0_orig, w_orig, counts, bin_start, sorted_l, i0_sorted, w_sorted, s);
  }
  if (e == cudaSuccess)
    e = launch_spread(reinterpret_cast<const float2*>(d_phasor), F, bin_start, sorted_l, i0_sorted, w_sorted, w,
                      tiles, W, fine, s);
  const int logf = 31 - __builtin_clz((unsigned)nf);
  PanelArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.scale = 1.f;
  pa.CHI = 1;
  pa.hi_total = 1;
  pa.in_slo = 1;
  pa.out_slo = 1;
  pa.lo_total = F;
  pa.CLO = panel_width(logf);
  pa.twiddle = tw;
  if (e == cudaSuccess) {  // FFT along x of every window row, keep kx in I_M
    PanelArgs a = pa;
    a.in = fine;
    a.out = R1;
    a.in_sb = (long long)W * F;
    a.in_si = F;
    a.out_sb = (long long)M * F;
    a.out_si = F;
    a.nin = W;
    a.in_off = g0;
    a.nout = M;
    a.out_off = -M / 2;
    a.batch = W;
    e = launch_panel_fft(logf, false, a, s);
  }
  if (e == cudaSuccess) {  // FFT along y of every kx column, keep ky in I_M, divide by psi_hat(kx) psi_hat(ky)
    PanelArgs a = pa;
    a.in = R1;
    a.out = reinterpret_cast<float2*>(d_spectrum);
    a.in_sb = F;
    a.in_si = (long long)M * F;
    a.out_sb = F;
    a.out_si = (long long)M * F;
    a.nin = W;
    a.in_off = g0;
    a.nout = M;
    a.out_off = -M / 2;
    a.batch = M;
    a.mul_o = dec;
    a.mul_b = dec;
    e = launch_panel_fft(logf, false, a, s);
  }
  return from_cuda(e);
}
