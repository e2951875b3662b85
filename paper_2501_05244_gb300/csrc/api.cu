// C ABI of libnursd: plan lifecycle, argument validation and the launch
// sequences of each entry point (see include/nursd.h for the contract).
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_fp16.h>

#include "nursd_internal.cuh"

using namespace nursd;

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kC = 299792458.0;  // speed of light [m/s]

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(long long v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
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
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Test hook (nursd_test_fail_allocation): the device allocation that brings the countdown to zero fails.
std::atomic<int> g_alloc_countdown{-1};

// cudaMalloc, unless the test hook makes this allocation fail.
cudaError_t dev_malloc(void** ptr, size_t bytes) {
  int c = g_alloc_countdown.load();
  while (c > 0 && !g_alloc_countdown.compare_exchange_weak(c, c - 1)) {
  }
  if (c == 1) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

// ES kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| < 1.
double es_kernel(double z, double beta) { return std::fabs(z) < 1.0 ? std::exp(beta * (std::sqrt(1.0 - z * z) - 1.0)) : 0.0; }

}  // namespace

// The per-call workspace of the point sort, the type-1 passes and the inverse passes.  The batched form
// keeps one per concurrent stream and swaps it into the plan while it enqueues that stream's launches
// (launches read the pointers when they are enqueued).
struct Workspace {
  int* bin_of = nullptr;
  int2* i0_orig = nullptr;
  int* slot_of = nullptr;
  float* w_orig = nullptr;
  int* counts = nullptr;
  int* bin_start = nullptr;
  int* sorted_l = nullptr;
  int2* i0_sorted = nullptr;
  float* w_sorted = nullptr;
  float2* frac_orig = nullptr;
  float2* frac_sorted = nullptr;
  float2* fine = nullptr;
  float2* R1 = nullptr;
  float2* T1 = nullptr;
};

constexpr int kMaxBatchStreams = 16;

struct nursd_plan_s {
  int device = 0;
  // tunables (nursd_plan_tune): spread tile height; streams of the batched form
  int spread_rows = 8;
  int batch_streams = 4;
  int batch_grouped = 1;
  int batch_tensor = 1;  // the batched contraction on the tensor cores where supported
  int contract_tc = 0;   // the single-reconstruction contraction (and its adjoint) on the tensor cores (opt-in)
  int group_size = 0;  // items per grouped launch (1 .. group; 0 until the workspaces exist)
  // geometry
  int N = 0, M = 0, nf = 0, Z = 0, F = 0, T = 0, w = 0, W = 0, tiles = 0, g0 = 0, ncls = 0, maxL = 0, L = -1;
  double pitch = 0, cx = 0, cy = 0, t0 = 0, dt = 0;
  float beta = 0;
  uint32_t flags = 0;
  std::vector<double> depths, omega, weight;
  // tables
  float2* twiddle = nullptr;
  float* deconv = nullptr;
  int2* cls = nullptr;
  float2* Gc = nullptr;
  float2* GcT = nullptr;  // transposed table [ncls][Z][F] for the adjoint (NURSD_ENABLE_ADJOINT)
  // position gradients (NURSD_ENABLE_ADJOINT): deconv_k[i] = (i - M/2) deconv[i], and the type-2
  // grids [W][W][F] of kx R and ky R
  float* deconv_k = nullptr;
  float2 *fine_dx = nullptr, *fine_dy = nullptr;
  __half* Bth = nullptr;  // temporal twiddles B^T [2F][T] (unit modulus), fp16 head
  __half* Btl = nullptr;  // and tail (B - head)
  float* wcol = nullptr;  // weight of each temporal output column [2F] (w_f twice)
  TemporalFix tfix{};     // rows outside the fp16 split's window, recomputed scaled
  TemporalMaps tmaps{};   // TMA descriptors of Bth/Btl for the tcgen05 form (ok = 0: mma.sync form)
  // SRSD tables (h_srsd_pitch given): scaled transfer table [Z][ncls][F], chirps [Z][M], FFT(b)/(2M) [Z][2M]
  std::vector<double> srsd_pitch;
  std::vector<double> srsd_scale;  // srsd_pitch / pitch (host copy of srsd_scale_d)
  double* srsd_scale_d = nullptr;  // device [Z]
  // SRSD depths with scale >= 1 take the scaled DFT by interpolation of one oversampled spectrum:
  // si_yh [2M][2M][F], its half-transformed rows si_scr [M][2M][F], and per depth the first tap
  // m0 [M] and weights [M][w] of the coordinates 2 kappa / s
  float2 *si_yh = nullptr, *si_scr = nullptr;
  int* si_m0 = nullptr;
  float* si_wt = nullptr;
  std::vector<char> si_interp;
  bool si_any = false;
  int* si_zlist = nullptr;  // device list of the interpolated depths (one launch covers them all)
  int si_nz = 0;
  // NU-SFFT (srsd_forward_nonuniform), built on first use: 1 / psi_hat(g) over the spread window [W],
  // taps [Z][M] / [Z][M][w] at kappa / s_z on the 2M grid (1 / psi_hat(kappa / s_z) folded into the
  // weights), the half-transformed window rows [W][2M][F] and the list of every depth
  float* nu_dec_w = nullptr;
  int* nu_m0 = nullptr;
  float* nu_wt = nullptr;
  float2* nu_rows = nullptr;
  int* nu_zlist = nullptr;
  bool nu_ready = false;
  std::vector<float> nu_host_f;
  std::vector<int> nu_host_i;
  // 3D NURSD (nursd_enable_3d): Mz z offsets of pitch dz, the window of Wz fine z cells from gz0, the 3D
  // transfer table [M][M][Mz][F], 1 / psi_hat_z [Mz], the slices' spectra [Wz][M][M][F], the 3D spectrum
  // [M][M][Mz][F], the plane's spectrum [M][M][F] and lattice field [F][N][N], a half transform [N][M][F],
  // the slice phasors [maxL][F] and the samples' fine z coordinates [maxL] (slot order)
  int nd_Mz = 0, nd_Wz = 0, nd_gz0 = 0;
  int nd_G = 0;  // z slices per group of stage 1's slice launches (their phasors, windows and rows side by side)
  float2 *nd_fine = nullptr, *nd_R1 = nullptr;
  double nd_dz = 0.0;
  float2 *nd_G3 = nullptr, *nd_U3w = nullptr, *nd_U3 = nullptr, *nd_What = nullptr, *nd_field = nullptr;
  float2 *nd_T = nullptr, *nd_Pz = nullptr;
  float *nd_decz = nullptr, *nd_uz = nullptr;
  bool nd_points = false;  // the current points carry heights (nursd_set_points_3d)
  std::vector<float> nd_host;
  float2* Gs = nullptr;
  float2* chirp = nullptr;
  float2* bhat = nullptr;
  // batched reconstructions (max_batch > 0): per-item phasors, spectra and depth spectra
  int maxB = 0;
  float2* phasor_all = nullptr;  // [maxB][maxL][F]
  float2* U_all = nullptr;       // [maxB][M][M][F]
  float2* Y_all = nullptr;       // [maxB][M][M][Z]
  int* counter = nullptr;
  // points
  int* bin_of = nullptr;
  int2* i0_orig = nullptr;
  int* slot_of = nullptr;  // sorted slot of each sample (inverse of sorted_l)
  float* w_orig = nullptr;
  int* counts = nullptr;
  int* bin_start = nullptr;
  int* sorted_l = nullptr;
  int2* i0_sorted = nullptr;
  float* w_sorted = nullptr;
  float2* frac_orig = nullptr;
  float2* frac_sorted = nullptr;
  // workspace
  float2* phasor = nullptr;
  float2* fine = nullptr;
  float2* R1 = nullptr;
  float2* U = nullptr;
  float2* Y = nullptr;
  float2* T1 = nullptr;
  int* status = nullptr;
  int64_t bytes = 0;
  std::vector<void*> allocs;
  // profiling: per stage, a list of (start, stop) events and how many are in use
  bool profiling = false;
  uint32_t profile_mask = 0;  // stages recorded while profiling
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[NURSD_NUM_STAGES];
  size_t ev_used[NURSD_NUM_STAGES] = {};
  int64_t launches = 0;

  template <class T>
  bool alloc(T*& p, size_t count) {
    if (count == 0) count = 1;
    void* q = nullptr;
    if (dev_malloc(&q, sizeof(T) * count) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(q);
    bytes += (int64_t)(sizeof(T) * count);
    p = static_cast<T*>(q);
    return true;
  }
  // per-frequency forms (nursd_forward_illuminated / nursd_transient_frames), allocated on first
  // use: pf_zg depths per group, products [M][M][zg F], half inverse [M][N][zg F], per-frequency
  // volumes [zg F][N][N], k_f / 2 pi [F] and depths [Z] in FP64, the frames' weights [T][F]
  int pf_zg = 0;
  float2 *pf_Y = nullptr, *pf_T = nullptr, *pf_V = nullptr, *pf_A = nullptr;
  double *pf_kap = nullptr, *pf_depth = nullptr;
  int pf_A_cap = 0;
  bool pf_equispaced = false;
  double pf_dkap = 0.0;
  std::vector<float2> pf_A_host;
  std::vector<double> pf_kap_host;
  // side stream of nursd_reconstruct (the point sort runs there, beside the temporal transform)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // batched form: `group` item workspaces side by side (gws: item b's arrays at b times the strides
  // below), used together by the batched launches and one per stream by the per-item form; the
  // streams 1 .. kMaxBatchStreams - 1 of that form (stream 0 is the caller's) and fork / join events
  int group = 0;
  Workspace gws;
  struct ItemStrides {
    size_t pts = 0, wts = 0, counts = 0, bins = 0, fine = 0, R1 = 0, T1 = 0;
  } gst;
  Workspace group_item(int b) const {
    Workspace w;
    w.bin_of = gws.bin_of + b * gst.pts;
    w.i0_orig = gws.i0_orig + b * gst.pts;
    w.slot_of = gws.slot_of + b * gst.pts;
    w.w_orig = gws.w_orig + b * gst.wts;
    w.counts = gws.counts + b * gst.counts;
    w.bin_start = gws.bin_start + b * gst.bins;
    w.sorted_l = gws.sorted_l + b * gst.pts;
    w.i0_sorted = gws.i0_sorted + b * gst.pts;
    w.w_sorted = gws.w_sorted + b * gst.wts;
    w.frac_orig = gws.frac_orig + b * gst.pts;
    w.frac_sorted = gws.frac_sorted + b * gst.pts;
    w.fine = gws.fine + b * gst.fine;
    w.R1 = gws.R1 + b * gst.R1;
    w.T1 = gws.T1 + b * gst.T1;
    return w;
  }
  cudaStream_t bstream[kMaxBatchStreams] = {};
  cudaEvent_t bev_fork = nullptr, bev_join[kMaxBatchStreams] = {};
  Workspace own() const {
    Workspace w;
    w.bin_of = bin_of;
    w.i0_orig = i0_orig;
    w.slot_of = slot_of;
    w.w_orig = w_orig;
    w.counts = counts;
    w.bin_start = bin_start;
    w.sorted_l = sorted_l;
    w.i0_sorted = i0_sorted;
    w.w_sorted = w_sorted;
    w.frac_orig = frac_orig;
    w.frac_sorted = frac_sorted;
    w.fine = fine;
    w.R1 = R1;
    w.T1 = T1;
    return w;
  }
  void use(const Workspace& w) {
    bin_of = w.bin_of;
    i0_orig = w.i0_orig;
    slot_of = w.slot_of;
    w_orig = w.w_orig;
    counts = w.counts;
    bin_start = w.bin_start;
    sorted_l = w.sorted_l;
    i0_sorted = w.i0_sorted;
    w_sorted = w.w_sorted;
    frac_orig = w.frac_orig;
    frac_sorted = w.frac_sorted;
    fine = w.fine;
    R1 = w.R1;
    T1 = w.T1;
  }
  ~nursd_plan_s() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
    if (bev_fork) cudaEventDestroy(bev_fork);
    for (int k = 0; k < kMaxBatchStreams; ++k) {
      if (bev_join[k]) cudaEventDestroy(bev_join[k]);
      if (bstream[k]) cudaStreamDestroy(bstream[k]);
    }
    for (auto& v : ev)
      for (auto& e : v) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {

// Records a stage's start/stop events on the launching stream while profiling is on.
class StageTimer {
 public:
  StageTimer(nursd_plan_s* p, int stage, cudaStream_t s, int launches) : p_(p), stage_(stage), s_(s) {
    p->launches += launches;
    if (!p->profiling || !(p->profile_mask & (1u << stage))) return;
    auto& v = p->ev[stage];
    if (p->ev_used[stage] == v.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
      if (cudaEventCreate(&e.first) != cudaSuccess || cudaEventCreate(&e.second) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
      v.push_back(e);
    }
    pair_ = &v[p->ev_used[stage]++];
    record(pair_->first);
  }
  ~StageTimer() {
    if (pair_) record(pair_->second);
  }

 private:
  nursd_plan_s* p_;
  int stage_;
  cudaStream_t s_;
  std::pair<cudaEvent_t, cudaEvent_t>* pair_ = nullptr;
  // an event-record node of the graph while s is being captured, a plain record otherwise
  void record(cudaEvent_t e) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s_, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(e, s_, cudaEventRecordExternal);
    else
      cudaEventRecord(e, s_);
  }
};

}  // namespace

namespace {

int from_cuda(cudaError_t e) { return e == cudaSuccess ? NURSD_OK : NURSD_ERR_CUDA; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// C[L][2F] = H[L][T] B diag(w): tcgen05 form when the plan has its descriptors and both buffers
// are 16-byte aligned, mma.sync form otherwise; each issues a first launch and a gather launch of
// the rows outside the fp16 split's window.  row_slot (optional): row l goes to row row_slot[l].
constexpr int kTemporalLaunches = 2;
cudaError_t run_temporal(const nursd_plan_s* p, const float* h, float* C, int L, cudaStream_t s,
                         const int* row_slot = nullptr) {
  if (p->tmaps.ok && aligned(h, 16) && aligned(C, 16))
    return launch_temporal_umma(p->tmaps, h, p->wcol, C, L, p->T, 2 * p->F, p->tfix, p->status, s, row_slot);
  return launch_temporal_tc(h, p->Bth, p->Btl, p->wcol, C, L, p->T, 2 * p->F, p->tfix, s, row_slot);
}

PanelArgs panel_base(const nursd_plan_s* p) {
  PanelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.scale = 1.f;
  a.CHI = 1;
  a.hi_total = 1;
  a.batch = 1;
  a.twiddle = p->twiddle;
  return a;
}

// Channel-last 1-D pass along an axis of length n_axis (window nin at offset in_off,
// nout bins at out_off), for C contiguous channels and `batch` items, optionally for nhi blocks of
// them at in_shi / out_shi.
cudaError_t axis_pass(const nursd_plan_s* p, const float2* in, float2* out, int logn, bool inv, int C, int batch,
                      long long in_sb, long long in_si, long long out_sb, long long out_si, int nin, int in_off,
                      int nout, int out_off, const float* mul_o, const float* mul_b, float scale, cudaStream_t s,
                      int nhi = 1, long long in_shi = 0, long long out_shi = 0) {
  PanelArgs a = panel_base(p);
  a.in = in;
  a.out = out;
  a.hi_total = nhi;  // an outer channel index (the items of a batched call), one per panel
  a.in_shi = in_shi;
  a.out_shi = out_shi;
  a.in_sb = in_sb;
  a.in_si = in_si;
  a.in_slo = 1;
  a.out_sb = out_sb;
  a.out_si = out_si;
  a.out_slo = 1;
  a.nin = nin;
  a.in_off = in_off;
  a.nout = nout;
  a.out_off = out_off;
  a.lo_total = C;
  a.CLO = panel_width(logn);
  a.batch = batch;
  a.mul_o = mul_o;
  a.mul_b = mul_b;
  a.scale = scale;
  return launch_panel_fft(logn, inv, a, s);
}

// Builds Ghat_{z,f} = DFT_M[exp(i k_f r)/r] for every depth in z-batches (FP64 phase, panel FFTs)
// and compresses it by symmetry class.  srsd = false: lattice pitch delta, into Gc (and GcT);
// srsd = true: pitch s_z delta per depth, into the depth-major SRSD table Gs.
int build_table(nursd_plan_s* p, bool srsd, cudaStream_t s) {
  const int M = p->M, F = p->F, Z = p->Z;
  const long long per_depth = (long long)M * M * F;
  int ZB = (int)std::max<long long>(1, (1LL << 28) / per_depth);  // ~2 GiB per buffer at most
  ZB = std::min(ZB, Z);
  float2 *g = nullptr, *tmp = nullptr;
  double *dz = nullptr, *dk = nullptr, *dp = nullptr;
  int rc = NURSD_OK;
  if (dev_malloc((void**)&g, sizeof(float2) * per_depth * ZB) != cudaSuccess ||
      dev_malloc((void**)&tmp, sizeof(float2) * per_depth * ZB) != cudaSuccess ||
      dev_malloc((void**)&dz, sizeof(double) * Z) != cudaSuccess ||
      dev_malloc((void**)&dk, sizeof(double) * F) != cudaSuccess ||
      dev_malloc((void**)&dp, sizeof(double) * Z) != cudaSuccess) {
    cudaGetLastError();
    rc = NURSD_ERR_OOM;
  }
  // wavenumbers of the kernel e^{ikr}/r; a confocal round trip doubles them
  const double kmul = (p->flags & NURSD_CONFOCAL) ? 2.0 : 1.0;
  std::vector<double> k(F);
  for (int f = 0; f < F; ++f) k[f] = kmul * p->omega[f] / kC;
  if (rc == NURSD_OK) {
    rc = from_cuda(cudaMemcpyAsync(dz, p->depths.data(), sizeof(double) * Z, cudaMemcpyHostToDevice, s));
    if (rc == NURSD_OK) rc = from_cuda(cudaMemcpyAsync(dk, k.data(), sizeof(double) * F, cudaMemcpyHostToDevice, s));
    if (rc == NURSD_OK && srsd)
      rc = from_cuda(cudaMemcpyAsync(dp, p->srsd_pitch.data(), sizeof(double) * Z, cudaMemcpyHostToDevice, s));
  }
  const int logM = ilog2(M);
  for (int z0 = 0; rc == NURSD_OK && z0 < Z; z0 += ZB) {
    const int zb = std::min(ZB, Z - z0);
    const int C = zb * F;
    rc = from_cuda(launch_gtf_generate(g, M, p->pitch, dz + z0, zb, dk, F, s, srsd ? dp + z0 : nullptr));
    if (rc == NURSD_OK)  // along jx, for each row jy
      rc = from_cuda(axis_pass(p, g, tmp, logM, false, C, M, (long long)M * C, C, (long long)M * C, C, M, -M / 2, M,
                               -M / 2, nullptr, nullptr, 1.f, s));
    if (rc == NURSD_OK)  // along jy, for each column kx
      rc = from_cuda(axis_pass(p, tmp, g, logM, false, C, M, C, (long long)M * C, C, (long long)M * C, M, -M / 2, M,
                               -M / 2, nullptr, nullptr, 1.f, s));
    if (rc == NURSD_OK) {
      if (srsd)
        rc = from_cuda(launch_gtf_compress_depthmajor(g, p->cls, p->ncls, M, F, zb, z0, p->Gs, s));
      else
        rc = from_cuda(launch_gtf_compress(g, p->cls, p->ncls, M, F, zb, Z, z0, p->Gc, p->GcT, s));
    }
  }
  if (rc == NURSD_OK) rc = from_cuda(cudaStreamSynchronize(s));
  cudaFree(g);
  cudaFree(tmp);
  cudaFree(dz);
  cudaFree(dk);
  cudaFree(dp);
  return rc;
}

// SRSD chirps c_z(n) = exp(-pi i n^2 / (M s_z)) on I_M and bhat_z = FFT_2M[b_z] / (2M) with
// b_z(d) = exp(+pi i d^2 / (M s_z)), |d| < M, placed at d mod 2M (phases in FP64).
int build_srsd_chirps(nursd_plan_s* p, cudaStream_t s) {
  const int M = p->M, Z = p->Z, L2 = 2 * M;
  std::vector<float2> ch((size_t)Z * M), b((size_t)Z * L2, make_float2(0.f, 0.f));
  for (int z = 0; z < Z; ++z) {
    const double sc = p->srsd_pitch[z] / p->pitch;
    for (int i = 0; i < M; ++i) {
      const double n = i - M / 2;
      const double ph = std::fmod(kPi * n * n / (M * sc), 2.0 * kPi);
      ch[(size_t)z * M + i] = make_float2((float)std::cos(ph), (float)-std::sin(ph));
    }
    for (int d = -(M - 1); d <= M - 1; ++d) {
      const double ph = std::fmod(kPi * (double)d * d / (M * sc), 2.0 * kPi);
      b[(size_t)z * L2 + ((d + L2) % L2)] = make_float2((float)std::cos(ph), (float)std::sin(ph));
    }
  }
  float2* db = nullptr;
  if (dev_malloc((void**)&db, sizeof(float2) * b.size()) != cudaSuccess) {
    cudaGetLastError();
    return NURSD_ERR_OOM;
  }
  p->srsd_scale.resize(Z);
  for (int z = 0; z < Z; ++z) p->srsd_scale[z] = p->srsd_pitch[z] / p->pitch;
  // interpolated depths: coordinate u = 2 kappa / s on the 2M-point grid, taps m0 .. m0 + w - 1 with
  // ES weights phi(2 (m - u) / w) in FP64 (the same kernel and beta as the spatial NUFFT)
  std::vector<int> m0v;
  std::vector<float> wtv;
  if (p->si_any) {
    const int w = p->w;
    const double beta = p->beta;  // the kernel whose transform the deconvolution table inverts
    m0v.assign((size_t)Z * M, 0);
    wtv.assign((size_t)Z * M * w, 0.f);
    for (int z = 0; z < Z; ++z) {
      if (!p->si_interp[z]) continue;
      for (int i = 0; i < M; ++i) {
        const double u = 2.0 * (i - M / 2) / p->srsd_scale[z];
        const int m0 = (int)std::ceil(u - 0.5 * w);
        m0v[(size_t)z * M + i] = m0;
        for (int t = 0; t < w; ++t) wtv[((size_t)z * M + i) * w + t] = (float)es_kernel(2.0 * (m0 + t - u) / w, beta);
      }
    }
  }
  std::vector<int> zl;
  for (int z = 0; z < Z && p->si_any; ++z)
    if (p->si_interp[z]) zl.push_back(z);
  p->si_nz = (int)zl.size();
  if (!zl.empty() && !p->si_zlist && !p->alloc(p->si_zlist, (size_t)Z)) {
    cudaFree(db);
    return NURSD_ERR_OOM;
  }
  int rc = from_cuda(cudaMemcpyAsync(p->chirp, ch.data(), sizeof(float2) * ch.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK && !zl.empty())
    rc = from_cuda(cudaMemcpyAsync(p->si_zlist, zl.data(), sizeof(int) * zl.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK)
    rc = from_cuda(
        cudaMemcpyAsync(p->srsd_scale_d, p->srsd_scale.data(), sizeof(double) * Z, cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK && p->si_any)
    rc = from_cuda(cudaMemcpyAsync(p->si_m0, m0v.data(), sizeof(int) * m0v.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK && p->si_any)
    rc = from_cuda(cudaMemcpyAsync(p->si_wt, wtv.data(), sizeof(float) * wtv.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK) rc = from_cuda(cudaMemcpyAsync(db, b.data(), sizeof(float2) * b.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK) {  // FFT of each depth's contiguous row of 2M values
    const int logL = ilog2(L2);
    PanelArgs a = panel_base(p);
    a.in = db;
    a.out = p->bhat;
    a.in_sb = L2;
    a.in_si = 1;
    a.in_slo = 1;
    a.out_sb = L2;
    a.out_si = 1;
    a.out_slo = 1;
    a.load_i_fastest = 1;
    a.store_o_fastest = 1;
    a.nin = L2;
    a.nout = L2;
    a.lo_total = 1;
    a.CLO = panel_width(logL);
    a.batch = Z;
    a.scale = 1.f / (float)L2;
    rc = from_cuda(launch_panel_fft(logL, false, a, s));
  }
  if (rc == NURSD_OK) rc = from_cuda(cudaStreamSynchronize(s));
  cudaFree(db);
  return rc;
}

// phasor rows in sample order, or (slot_ordered) already in the spread's sorted order.
int run_nufft1(nursd_plan_s* p, const float2* phasor, float2* spec, cudaStream_t s, bool slot_ordered = false) {
  const int F = p->F, M = p->M, W = p->W;
  const int logf = ilog2(p->nf);
  cudaError_t e;
  {
    StageTimer t(p, NURSD_STAGE_SPREAD, s, 1);
    SpreadItems one;
    one.status = p->status;
    e = launch_spread(phasor, F, p->bin_start, slot_ordered ? nullptr : p->sorted_l, p->i0_sorted, p->w_sorted, p->w,
                      p->tiles, W, p->fine, s, p->spread_rows, one);
  }
  if (e == cudaSuccess) {  // FFT along x of every window row, keep kx in I_M
    StageTimer t(p, NURSD_STAGE_FFT_X, s, 1);
    e = axis_pass(p, p->fine, p->R1, logf, false, F, W, (long long)W * F, F, (long long)M * F, F, W, p->g0, M, -M / 2,
                  nullptr, nullptr, 1.f, s);
  }
  if (e == cudaSuccess) {  // FFT along y of every kx column, keep ky in I_M, divide by psi_hat(kx) psi_hat(ky)
    StageTimer t(p, NURSD_STAGE_FFT_Y, s, 1);
    e = axis_pass(p, p->R1, spec, logf, false, F, M, F, (long long)M * F, F, (long long)M * F, W, p->g0, M, -M / 2,
                  p->deconv, p->deconv, 1.f, s);
  }
  return from_cuda(e);
}

// The second of the two pruned inverse passes: T [M][N][C] (ky, mx, c) -> out[c][my][mx], the
// inverse FFT along ky for every (mx, c) with my kept in I_N and the M^-2 scale; complex, or |.|.
// batch > 1: items b < batch of T at b in_sb, written at out + b out_sb (elements of the output type).
cudaError_t idft_crop_y(nursd_plan_s* p, const float2* T, int C, void* out, bool mag, cudaStream_t s, int batch = 1,
                        long long in_sb = 0, long long out_sb = 0) {
  const int M = p->M, N = p->N;
  const int logM = ilog2(M);
  cudaError_t e;
  {
    StageTimer t(p, NURSD_STAGE_IFFT_Y, s, 1);
    PanelArgs a = panel_base(p);
    a.in = T;
    a.in_si = (long long)N * C;
    a.in_shi = C;
    a.in_slo = 1;
    if (mag)
      a.out_mag = static_cast<float*>(out);
    else
      a.out = static_cast<float2*>(out);
    a.out_si = N;
    a.out_shi = 1;
    a.out_slo = (long long)N * N;
    a.nin = M;
    a.in_off = -M / 2;
    a.nout = N;
    a.out_off = -N / 2;
    a.hi_total = N;
    a.lo_total = C;
    const int cp = panel_width(logM);
    a.CLO = C >= 4 ? 4 : (C >= 2 ? 2 : 1);
    a.CHI = cp / a.CLO;
    a.scale = 1.f / ((float)M * (float)M);
    a.store_hi_fastest = 1;
    a.batch = batch;
    a.in_sb = in_sb;
    a.out_sb = out_sb;
    e = launch_panel_fft(logM, true, a, s);
  }
  return e;
}

// out[c][my][mx] = M^-2 sum_k Ysrc[k][c] e^{+2 pi i k.m / M} on I_N^2 for C channels (two pruned
// inverse passes through T [M][N][C]); out is complex, or |.| when mag.
cudaError_t idft_crop(nursd_plan_s* p, const float2* Ysrc, int C, float2* T, void* out, bool mag, cudaStream_t s) {
  const int M = p->M, N = p->N;
  const int logM = ilog2(M);
  cudaError_t e;
  {  // inverse FFT along kx, keep mx in I_N
    StageTimer t(p, NURSD_STAGE_IFFT_X, s, 1);
    e = axis_pass(p, Ysrc, T, logM, true, C, M, (long long)M * C, C, (long long)N * C, C, M, -M / 2, N, -N / 2,
                  nullptr, nullptr, 1.f, s);
  }
  if (e == cudaSuccess) e = idft_crop_y(p, T, C, out, mag, s);
  return e;
}

// V[z][my][mx] = M^-2 sum_k Y[k][z] e^{+2 pi i k.m / M} on I_N^2 (two pruned inverse passes).
int run_idft_crop(nursd_plan_s* p, void* out, cudaStream_t s, const float2* Ysrc = nullptr) {
  return from_cuda(idft_crop(p, Ysrc ? Ysrc : p->Y, p->Z, p->T1, out, (p->flags & NURSD_OUTPUT_MAGNITUDE) != 0, s));
}

// Y[k][z] = sum_f spec[k][f] G[cls(k)][f][z]: the FP32 bulk-copy form on Gc, or, when the plan opts in
// and keeps the transposed table (adjoint plans), the tensor-core form with GcT as the A operand.
cudaError_t contract_forward(nursd_plan_s* p, const float2* spec, cudaStream_t s) {
  if (p->contract_tc && p->GcT && contract_tc_supported(p->M, p->Z, p->F))
    return launch_contract_tc(spec, p->GcT, p->cls, p->ncls, p->M, p->Z, p->F, false, p->Y, s, p->status);
  return launch_contract(spec, p->Gc, p->cls, p->ncls, p->M, p->F, p->Z, p->Y, s, p->status);
}

int run_propagate(nursd_plan_s* p, const float2* spec, void* out, cudaStream_t s) {
  cudaError_t e;
  {
    StageTimer t(p, NURSD_STAGE_CONTRACT, s, 1);
    e = contract_forward(p, spec, s);
  }
  if (e != cudaSuccess) return from_cuda(e);
  return run_idft_crop(p, out, s);
}

// Scaled spectra Y^S_z [M][M][Z] (into p->Y) from a NUFFT-1 spectrum U (in p->U): see srsd_forward in
// nursd.h.  Depths with scale >= 1 take the scaled DFT by ES interpolation of one oversampled spectrum
// (srsd_interp.cu); the others by Bluestein's chirp-z.
int run_srsd_spectra(nursd_plan_s* p, cudaStream_t s) {
  const int M = p->M, F = p->F, Z = p->Z;
  const int logM = ilog2(M), logL = logM + 1;
  cudaError_t e;
  {  // gridded input u = M^-2 IDFT_M[U]: along kx (rows ky), then along ky (columns nx)
    StageTimer t(p, NURSD_STAGE_SRSD, s, 2);
    e = axis_pass(p, p->U, p->R1, logM, true, F, M, (long long)M * F, F, (long long)M * F, F, M, -M / 2, M, -M / 2,
                  nullptr, nullptr, 1.f, s);
    if (e == cudaSuccess)
      e = axis_pass(p, p->R1, p->fine, logM, true, F, M, F, (long long)M * F, F, (long long)M * F, M, -M / 2, M,
                    -M / 2, nullptr, nullptr, 1.f / ((float)M * (float)M), s);
  }
  if (e == cudaSuccess && p->si_any) {  // oversampled spectrum of u / (psi_hat x psi_hat), shared by the
                                        // interpolated depths: FFT_2M along nx, then along ny
    StageTimer t(p, NURSD_STAGE_SRSD, s, 2);
    const int L = 2 * M;
    PanelArgs a = panel_base(p);  // u [ny][nx][F] -> si_scr [ny][mx][F]
    a.in = p->fine;
    a.in_sb = (long long)M * F;
    a.in_si = F;
    a.in_slo = 1;
    a.mul_i = p->deconv;  // 1 / psi_hat(n), window index i <-> n = i - M/2
    a.out = p->si_scr;
    a.out_sb = (long long)L * F;
    a.out_si = F;
    a.out_slo = 1;
    a.nin = M;
    a.in_off = -M / 2;
    a.nout = L;
    a.out_off = -L / 2;
    a.lo_total = F;
    a.CLO = panel_width(logL);
    a.batch = M;
    e = launch_panel_fft(logL, false, a, s);
    if (e == cudaSuccess) {  // si_scr columns -> si_yh [my][mx][F]
      PanelArgs b = a;
      b.in = p->si_scr;
      b.in_sb = F;
      b.in_si = (long long)L * F;
      b.out = p->si_yh;
      b.out_sb = F;
      b.out_si = (long long)L * F;
      b.batch = L;
      e = launch_panel_fft(logL, false, b, s);
    }
  }
  if (e == cudaSuccess && p->si_any && srsd_interp_adds(F, 2 * M, p->w))  // channel halves are added into a zeroed Y
    e = cudaMemsetAsync(p->Y, 0, sizeof(float2) * (size_t)M * M * Z, s);
  if (e == cudaSuccess && p->si_any) {  // every depth with scale >= 1: taps and contraction, one launch
    StageTimer t(p, NURSD_STAGE_SRSD, s, 1);
    e = launch_srsd_interp_xy_contract(p->si_yh, 2 * M, M, F, Z, p->si_zlist, p->si_nz, p->w, p->si_m0, p->si_wt,
                                       p->Gs, p->ncls, p->Y, p->status, s);
  }
  for (int z = 0; e == cudaSuccess && z < Z; ++z) {
    if (p->si_interp[z]) continue;
    StageTimer t(p, NURSD_STAGE_SRSD, s, 3);
    const float2* ch = p->chirp + (size_t)z * M;
    const float2* bh = p->bhat + (size_t)z * 2 * M;
    PanelArgs a = panel_base(p);  // scaled DFT along nx for every (ny, f): u -> Q [ny][kx'][F]
    a.in = p->fine;
    a.out = p->R1;
    a.in_sb = (long long)M * F;
    a.in_si = F;
    a.in_slo = 1;
    a.out_sb = (long long)M * F;
    a.out_si = F;
    a.out_slo = 1;
    a.nin = M;
    a.in_off = -M / 2;
    a.nout = M;
    a.out_off = -M / 2;
    a.lo_total = F;
    a.CLO = panel_width(logL);
    a.batch = M;
    e = launch_panel_bluestein(logL, a, ch, bh, ch, s);
    if (e == cudaSuccess) {  // scaled DFT along ny for every (kx', f): Q -> Phat [ky'][kx'][F]
      PanelArgs b = a;
      b.in = p->R1;
      b.out = p->U;
      b.in_sb = F;
      b.in_si = (long long)M * F;
      b.out_sb = F;
      b.out_si = (long long)M * F;
      e = launch_panel_bluestein(logL, b, ch, bh, ch, s);
    }
    if (e == cudaSuccess)
      e = launch_contract_depth(p->U, p->Gs + (size_t)z * p->ncls * F, p->cls, p->ncls, M, F, Z, z, p->Y, s);
  }
  return from_cuda(e);
}

// psi_hat(a) = (w / 2) int_{-1}^{1} phi(z) cos(pi a w z / nf) dz, the transform of the ES kernel spread over
// w cells of the nf-point fine grid, at a frequency or (for the dual interpolation) a spatial index a.
double es_transform(double a, int w, double beta, int nf) {
  static std::vector<double> gx, gw;
  if (gx.empty()) gauss_legendre(256, gx, gw);
  double s_ = 0.0;
  for (size_t j = 0; j < gx.size(); ++j) s_ += gw[j] * es_kernel(gx[j], beta) * std::cos(kPi * a * w * gx[j] / nf);
  return 0.5 * w * s_;
}

// Tables and workspace of the NU-SFFT, on first use; every depth must have scale >= 1.
int ensure_nusfft(nursd_plan_s* p, cudaStream_t s) {
  if (p->nu_ready) return NURSD_OK;
  if (!p->Gs || !p->si_yh) return NURSD_ERR_INVALID_ARG;
  const int M = p->M, Z = p->Z, w = p->w, W = p->W, nf = p->nf;
  for (int z = 0; z < Z; ++z)
    if (!(p->srsd_scale[z] >= 1.0)) return NURSD_ERR_UNSUPPORTED;
  if (!p->nu_m0 &&  // first use (the buffers stay when new SRSD pitches only change the taps)
      !(p->alloc(p->nu_dec_w, W) && p->alloc(p->nu_m0, (size_t)Z * M) && p->alloc(p->nu_wt, (size_t)Z * M * w) &&
        p->alloc(p->nu_rows, (size_t)W * 2 * M * p->F) && p->alloc(p->nu_zlist, Z)))
    return NURSD_ERR_OOM;
  // host copies are plan-owned: the uploads below may complete after this call returns
  p->nu_host_f.assign((size_t)W + (size_t)Z * M * w, 0.f);
  p->nu_host_i.assign((size_t)Z * M + Z, 0);
  float* dec = p->nu_host_f.data();
  float* wt = dec + W;
  int* m0 = p->nu_host_i.data();
  int* zl = m0 + (size_t)Z * M;
  for (int i = 0; i < W; ++i) dec[i] = (float)(1.0 / es_transform(p->g0 + i, w, p->beta, nf));
  for (int z = 0; z < Z; ++z) {
    zl[z] = z;
    for (int i = 0; i < M; ++i) {
      const double nu = (i - M / 2) / p->srsd_scale[z];  // frequency on the nf = 2M grid
      const int a = (int)std::ceil(nu - 0.5 * w);
      const double inv = 1.0 / es_transform(nu, w, p->beta, nf);
      m0[(size_t)z * M + i] = a;
      for (int t = 0; t < w; ++t)
        wt[((size_t)z * M + i) * w + t] = (float)(es_kernel(2.0 * (a + t - nu) / w, p->beta) * inv);
    }
  }
  cudaError_t e = cudaMemcpyAsync(p->nu_dec_w, dec, sizeof(float) * W, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->nu_wt, wt, sizeof(float) * Z * M * w, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->nu_m0, m0, sizeof(int) * Z * M, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p->nu_zlist, zl, sizeof(int) * Z, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return NURSD_ERR_CUDA;
  p->nu_ready = true;
  return NURSD_OK;
}

// NU-SFFT spectra into p->Y from phasors in sample order: spread, FFT of the whole 2M x 2M grid of
// b / (psi_hat x psi_hat) (spatial deconvolution), then per depth the ES taps at kappa / s_z fused
// with the contraction.
int run_nusfft_spectra(nursd_plan_s* p, const float2* phasor, cudaStream_t s) {
  const int M = p->M, F = p->F, Z = p->Z, W = p->W, L2 = 2 * M;
  const int logL = ilog2(L2);
  cudaError_t e;
  {
    StageTimer t(p, NURSD_STAGE_SPREAD, s, 1);
    e = launch_spread(phasor, F, p->bin_start, p->sorted_l, p->i0_sorted, p->w_sorted, p->w, p->tiles, W, p->fine, s,
                      p->spread_rows);
  }
  if (e == cudaSuccess) {  // along x of every window row: [W][W][F] -> [W][2M][F]
    StageTimer t(p, NURSD_STAGE_SRSD, s, 2);
    PanelArgs a = panel_base(p);
    a.in = p->fine;
    a.in_sb = (long long)W * F;
    a.in_si = F;
    a.in_slo = 1;
    a.mul_i = p->nu_dec_w;  // 1 / psi_hat(g), window index i <-> g = g0 + i
    a.out = p->nu_rows;
    a.out_sb = (long long)L2 * F;
    a.out_si = F;
    a.out_slo = 1;
    a.nin = W;
    a.in_off = p->g0;
    a.nout = L2;
    a.out_off = -M;
    a.lo_total = F;
    a.CLO = panel_width(logL);
    a.batch = W;
    e = launch_panel_fft(logL, false, a, s);
    if (e == cudaSuccess) {  // along y of every column: [W][2M][F] -> [2M][2M][F]
      PanelArgs b = a;
      b.in = p->nu_rows;
      b.in_sb = F;
      b.in_si = (long long)L2 * F;
      b.out = p->si_yh;
      b.out_sb = F;
      b.out_si = (long long)L2 * F;
      b.batch = L2;
      e = launch_panel_fft(logL, false, b, s);
    }
  }
  if (e == cudaSuccess && srsd_interp_adds(F, L2, p->w))
    e = cudaMemsetAsync(p->Y, 0, sizeof(float2) * (size_t)M * M * Z, s);
  if (e == cudaSuccess) {
    StageTimer t(p, NURSD_STAGE_SRSD, s, 1);
    e = launch_srsd_interp_xy_contract(p->si_yh, L2, M, F, Z, p->nu_zlist, Z, p->w, p->nu_m0, p->nu_wt, p->Gs,
                                       p->ncls, p->Y, p->status, s);
  }
  return from_cuda(e);
}

// The 3D transfer table Ghat3_f(k) = DFT_3[G(j delta, jz dz)], k in I_M^2 x I_Mz, stored [ky][kx][kz][f]:
// the kernel sampled on the offset grid (G = 0 at the zero offset), the lateral passes, then along jz.
int build_table_3d(nursd_plan_s* p, cudaStream_t s) {
  const int M = p->M, F = p->F, Mz = p->nd_Mz;
  const size_t n = (size_t)M * M * Mz * F;
  float2 *g = nullptr, *tmp = nullptr;
  double *djz = nullptr, *dk = nullptr;
  int rc = NURSD_OK;
  if (dev_malloc((void**)&g, sizeof(float2) * n) != cudaSuccess || dev_malloc((void**)&tmp, sizeof(float2) * n) != cudaSuccess ||
      dev_malloc((void**)&djz, sizeof(double) * Mz) != cudaSuccess || dev_malloc((void**)&dk, sizeof(double) * F) != cudaSuccess) {
    cudaGetLastError();
    rc = NURSD_ERR_OOM;
  }
  std::vector<double> jz(Mz), k(F);
  for (int i = 0; i < Mz; ++i) jz[i] = (i - Mz / 2) * p->nd_dz;
  const double kmul = (p->flags & NURSD_CONFOCAL) ? 2.0 : 1.0;
  for (int f = 0; f < F; ++f) k[f] = kmul * p->omega[f] / kC;
  if (rc == NURSD_OK) rc = from_cuda(cudaMemcpyAsync(djz, jz.data(), sizeof(double) * Mz, cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK) rc = from_cuda(cudaMemcpyAsync(dk, k.data(), sizeof(double) * F, cudaMemcpyHostToDevice, s));
  const int C = Mz * F, logM = ilog2(M);
  if (rc == NURSD_OK)  // g[jy][jx][jz F + f] with r = sqrt(|j delta|^2 + (jz dz)^2)
    rc = from_cuda(launch_gtf_generate(g, M, p->pitch, djz, Mz, dk, F, s));
  if (rc == NURSD_OK)  // the zero offset (index M/2, M/2, Mz/2), where r = 0: G = 0
    rc = from_cuda(cudaMemsetAsync(g + ((size_t)(M / 2) * M + M / 2) * C + (size_t)(Mz / 2) * F, 0,
                                   sizeof(float2) * F, s));
  if (rc == NURSD_OK)
    rc = from_cuda(axis_pass(p, g, tmp, logM, false, C, M, (long long)M * C, C, (long long)M * C, C, M, -M / 2, M,
                             -M / 2, nullptr, nullptr, 1.f, s));
  if (rc == NURSD_OK)
    rc = from_cuda(axis_pass(p, tmp, g, logM, false, C, M, C, (long long)M * C, C, (long long)M * C, M, -M / 2, M,
                             -M / 2, nullptr, nullptr, 1.f, s));
  if (rc == NURSD_OK)  // along jz for every lateral mode: [ky][kx][jz][f] -> [ky][kx][kz][f]
    rc = from_cuda(axis_pass(p, g, p->nd_G3, ilog2(Mz), false, F, M * M, C, F, C, F, Mz, -Mz / 2, Mz, -Mz / 2,
                             nullptr, nullptr, 1.f, s));
  if (rc == NURSD_OK) rc = from_cuda(cudaStreamSynchronize(s));
  cudaFree(g);
  cudaFree(tmp);
  cudaFree(djz);
  cudaFree(dk);
  return rc;
}

// Workspace of the per-frequency forms (see the plan members), allocated on first use.
int ensure_per_frequency(nursd_plan_s* p, cudaStream_t s) {
  if (p->pf_zg > 0) return NURSD_OK;
  const int M = p->M, N = p->N, F = p->F, Z = p->Z;
  // groups of 4 depths where the kx pass forms the products itself (radix-32 lengths); otherwise
  // as many depths as keep a group within 512 channels
  const bool fusable = Z % 4 == 0 && F % 2 == 0 && (M == 512 || M == 1024);
  const int zg = fusable ? 4 : std::max(1, std::min(Z, 512 / F));
  const size_t C = (size_t)zg * F;
  if (!(p->alloc(p->pf_Y, fusable ? 1 : (size_t)M * M * C) && p->alloc(p->pf_T, (size_t)M * N * C) &&
        p->alloc(p->pf_V, C * N * N) && p->alloc(p->pf_kap, F) && p->alloc(p->pf_depth, Z)))
    return NURSD_ERR_OOM;
  std::vector<double> kap(F);
  for (int f = 0; f < F; ++f) kap[f] = p->omega[f] / (2.0 * kPi * kC);
  const double dk = F > 1 ? (kap[F - 1] - kap[0]) / (F - 1) : 0.0;
  bool equi = true;
  for (int f = 0; f < F; ++f) equi = equi && std::fabs(kap[f] - (kap[0] + f * dk)) <= 1e-13 * std::fabs(kap[F - 1]);
  p->pf_equispaced = equi;
  p->pf_dkap = dk;
  // both host arrays are plan-owned and stay unchanged afterwards
  cudaError_t e = cudaMemcpyAsync(p->pf_depth, p->depths.data(), sizeof(double) * Z, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    p->pf_kap_host = kap;
    e = cudaMemcpyAsync(p->pf_kap, p->pf_kap_host.data(), sizeof(double) * F, cudaMemcpyHostToDevice, s);
  }
  if (e != cudaSuccess) return NURSD_ERR_CUDA;
  p->pf_zg = zg;
  return NURSD_OK;
}

// Per-frequency forms from the spectrum in p->U: for each group of pf_zg depths, the products
// U_f Ghat_{z,f}, the two pruned inverse passes over all zg*F channels, then the weighted sum over
// f -- by the illumination mask of *illum (frames == 0) or by exp(+i w_f t) for each of the
// `frames` times (weights already in p->pf_A).
int run_per_frequency(nursd_plan_s* p, const double* illum, int frames, float2* out, cudaStream_t s) {
  const int M = p->M, N = p->N, F = p->F, Z = p->Z, zg = p->pf_zg;
  IllumArgs ia;
  std::memset(&ia, 0, sizeof(ia));
  if (frames == 0) {
    ia.xp = illum[0];
    ia.yp = illum[1];
    ia.zp = illum[2];
    ia.cx = p->cx;
    ia.cy = p->cy;
    ia.pitch = p->pitch;
    ia.depth = p->pf_depth;
    ia.kap = p->pf_kap;
    ia.dkap = p->pf_dkap;
    ia.equispaced = p->pf_equispaced ? 1 : 0;
  }
  cudaError_t e = cudaSuccess;
  for (int z0 = 0; z0 < Z && e == cudaSuccess; z0 += zg) {
    const int n = std::min(zg, Z - z0), C = n * F;
    // groups of 4 depths on the radix-32 lengths form the products inside the kx pass's window
    // staging (channel 4 f + zz) instead of writing and re-reading them (channel zz F + f)
    const bool fused = n == 4 && Z % 4 == 0 && F % 2 == 0 && (M == 512 || M == 1024);
    if (fused) {
      PanelArgs a = panel_base(p);
      a.in = p->U;
      a.in_sb = (long long)M * F;
      a.in_si = F;
      a.in_slo = 1;
      a.prod_g = p->Gc;
      a.prod_F = F;
      a.prod_Z = Z;
      a.prod_z0 = z0;
      a.out = p->pf_T;
      a.out_sb = (long long)N * C;
      a.out_si = C;
      a.out_slo = 1;
      a.nin = M;
      a.in_off = -M / 2;
      a.nout = N;
      a.out_off = -N / 2;
      a.lo_total = C;
      a.CLO = panel_width(ilog2(M));
      a.batch = M;
      {
        StageTimer t(p, NURSD_STAGE_IFFT_X, s, 1);
        e = launch_panel_fft(ilog2(M), true, a, s);
      }
      if (e == cudaSuccess && frames == 0) {  // channel-last volumes [N][N][C] for the warp-per-voxel sum
        StageTimer t(p, NURSD_STAGE_IFFT_Y, s, 1);
        PanelArgs b = panel_base(p);
        b.in = p->pf_T;
        b.in_si = (long long)N * C;
        b.in_shi = C;
        b.in_slo = 1;
        b.out = p->pf_V;
        b.out_si = (long long)N * C;
        b.out_shi = C;
        b.out_slo = 1;
        b.nin = M;
        b.in_off = -M / 2;
        b.nout = N;
        b.out_off = -N / 2;
        b.hi_total = N;
        b.lo_total = C;
        b.CLO = panel_width(ilog2(M));
        b.scale = 1.f / ((float)M * (float)M);
        e = launch_panel_fft(ilog2(M), true, b, s);
      } else if (e == cudaSuccess) {
        e = idft_crop_y(p, p->pf_T, C, p->pf_V, false, s);
      }
    } else {
      {
        StageTimer t(p, NURSD_STAGE_PER_FREQUENCY, s, 1);
        e = launch_transfer_depths(p->U, p->Gc, M, F, Z, z0, n, p->pf_Y, s);
      }
      if (e == cudaSuccess) e = idft_crop(p, p->pf_Y, C, p->pf_T, p->pf_V, false, s);
    }
    const int cz = fused ? 1 : F, cf = fused ? n : 1;  // channel of (zz, f) = zz cz + f cf
    if (e == cudaSuccess) {
      StageTimer t(p, NURSD_STAGE_PER_FREQUENCY, s, 1);
      if (frames == 0)
        e = fused ? launch_illum_sum_cl(p->pf_V, F, N, z0, n, ia, out, s)
                  : launch_illum_sum(p->pf_V, F, N, z0, n, cz, cf, ia, out, s);
      else
        e = launch_frames_sum(p->pf_V, F, N, Z, z0, n, cz, cf, p->pf_A, frames, out, s);
    }
  }
  return from_cuda(e);
}

// Adjoint of run_propagate up to the spectrum: R[k][f] = sum_z conj(Ghat) * M^-2 DFT_M[pad V_z](k),
// V [Z][N][N] -> p->U [M][M][F].
int run_adjoint_spectrum(nursd_plan_s* p, const float2* vol, cudaStream_t s) {
  const int M = p->M, N = p->N, Z = p->Z, F = p->F;
  const int logM = ilog2(M);
  cudaError_t e;
  {  // DFT along mx of every (z, my) row (contiguous in memory), full kx in I_M
    StageTimer t(p, NURSD_STAGE_IFFT_Y, s, 1);
    PanelArgs a = panel_base(p);
    a.in = vol;
    a.in_sb = N;
    a.in_si = 1;
    a.in_slo = (long long)N * N;
    a.load_i_fastest = 1;
    a.out = p->T1;
    a.out_sb = (long long)M * Z;
    a.out_si = Z;
    a.out_slo = 1;
    a.nin = N;
    a.in_off = -N / 2;
    a.nout = M;
    a.out_off = -M / 2;
    a.lo_total = Z;
    a.CLO = panel_width(logM);
    a.batch = N;
    e = launch_panel_fft(logM, false, a, s);
  }
  if (e == cudaSuccess) {  // DFT along my for every kx, full ky, scaled by M^-2
    StageTimer t(p, NURSD_STAGE_IFFT_X, s, 1);
    e = axis_pass(p, p->T1, p->Y, logM, false, Z, M, Z, (long long)M * Z, Z, (long long)M * Z, N, -N / 2, M, -M / 2,
                  nullptr, nullptr, 1.f / ((float)M * (float)M), s);
  }
  if (e == cudaSuccess) {
    StageTimer t(p, NURSD_STAGE_CONTRACT, s, 1);
    if (p->contract_tc && contract_tc_supported(M, F, Z))  // U[k][f] = sum_z conj(Gc[c][f][z]) Y[k][z]
      e = launch_contract_tc(p->Y, p->Gc, p->cls, p->ncls, M, F, Z, true, p->U, s, p->status);
    else
      e = launch_contract_adjoint(p->Y, p->GcT, p->cls, p->ncls, M, F, Z, p->U, s, p->status);
  }
  return from_cuda(e);
}

// Type 2 from a spectrum [M][M][C] onto the fine window: divide by
// psi_hat(kx) psi_hat(ky) (folded into the first pass's input and batch
// factors), zero-pad to the fine grid, inverse FFT along kx, then along ky.
// plane_major = false: fine [W][W][C] (channel-last, for relay samples);
// plane_major = true: fine [C][W][W] (one plane per channel, for voxel sets).
// mul_kx / mul_ky (default: the deconvolution table) are the real factors of kx and ky, and
// fine_out (default: p->fine) the grid written.
int run_type2_to_fine(nursd_plan_s* p, const float2* spec, int C, bool plane_major, float scale, cudaStream_t s,
                      const float* mul_kx = nullptr, const float* mul_ky = nullptr, float2* fine_out = nullptr) {
  const int M = p->M, W = p->W;
  if (!mul_kx) mul_kx = p->deconv;
  if (!mul_ky) mul_ky = p->deconv;
  if (!fine_out) fine_out = p->fine;
  const int logf = ilog2(p->nf);
  cudaError_t e;
  {
    StageTimer t(p, NURSD_STAGE_FFT_Y, s, 1);
    PanelArgs a = panel_base(p);
    a.in = spec;
    a.in_sb = (long long)M * C;
    a.in_si = C;
    a.in_slo = 1;
    a.mul_i = mul_kx;  // 1/psi_hat(kx), input index i <-> kx = i - M/2
    a.mul_b = mul_ky;  // 1/psi_hat(ky), batch b <-> ky = b - M/2
    a.out = p->R1;
    a.out_sb = (long long)W * C;
    a.out_si = C;
    a.out_slo = 1;
    a.nin = M;
    a.in_off = -M / 2;
    a.nout = W;
    a.out_off = p->g0;
    a.lo_total = C;
    a.CLO = panel_width(logf);
    a.batch = M;
    e = launch_panel_fft(logf, true, a, s);
  }
  if (e == cudaSuccess) {
    StageTimer t(p, NURSD_STAGE_FFT_X, s, 1);
    PanelArgs a = panel_base(p);
    a.in = p->R1;
    a.nin = M;
    a.in_off = -M / 2;
    a.nout = W;
    a.out_off = p->g0;
    a.out = fine_out;
    a.scale = scale;
    const int cp = panel_width(logf);
    if (!plane_major) {  // batch over x, channels c
      a.in_sb = C;
      a.in_si = (long long)W * C;
      a.in_slo = 1;
      a.out_sb = C;
      a.out_si = (long long)W * C;
      a.out_slo = 1;
      a.lo_total = C;
      a.CLO = cp;
      a.batch = W;
    } else {  // channels (x, c), written as fine[c][y][x] with x fastest
      a.in_si = (long long)W * C;
      a.in_shi = C;
      a.in_slo = 1;
      a.out_si = W;
      a.out_shi = 1;
      a.out_slo = (long long)W * W;
      a.hi_total = W;
      a.lo_total = C;
      a.CLO = C >= 4 ? 4 : (C >= 2 ? 2 : 1);
      a.CHI = cp / a.CLO;
      a.store_hi_fastest = 1;
    }
    e = launch_panel_fft(logf, true, a, s);
  }
  return from_cuda(e);
}

int check_plan(nursd_plan_t p) { return p ? NURSD_OK : NURSD_ERR_INVALID_ARG; }

// SRSD buffers for the pitches in p->srsd_pitch (allocated on first use) and the choice of the
// interpolated depths (scale >= 1), with their workspace.
int alloc_srsd(nursd_plan_s* p) {
  const int M = p->M, w = p->w;
  if (!p->Gs && !(p->alloc(p->Gs, (size_t)p->ncls * p->F * p->Z) && p->alloc(p->chirp, (size_t)p->Z * M) &&
                  p->alloc(p->bhat, (size_t)p->Z * 2 * M) && p->alloc(p->srsd_scale_d, p->Z)))
    return NURSD_ERR_OOM;
  p->si_interp.assign(p->Z, 0);
  p->si_any = false;
  for (int z = 0; z < p->Z; ++z) {
    const double sc = p->srsd_pitch[z] / p->pitch;
    if (!(sc >= 1.0) || p->F > 256) continue;
    p->si_interp[z] = 1;
    p->si_any = true;
  }
  if (p->si_any && !p->si_yh) {
    const size_t L = 2 * (size_t)M;
    if (!(p->alloc(p->si_yh, L * L * p->F) && p->alloc(p->si_scr, M * L * p->F) &&
          p->alloc(p->si_m0, (size_t)p->Z * M) && p->alloc(p->si_wt, (size_t)p->Z * M * w)))
      return NURSD_ERR_OOM;
  }
  return NURSD_OK;
}

}  // namespace

extern "C" {

const char* nursd_status_string(int status) {
  switch (status) {
    case NURSD_OK: return "ok";
    case NURSD_ERR_INVALID_ARG: return "invalid argument";
    case NURSD_ERR_OOM: return "device out of memory";
    case NURSD_ERR_CUDA: return "CUDA error";
    case NURSD_ERR_TIMEOUT: return "bounded device wait timed out";
    case NURSD_ERR_UNSUPPORTED: return "unsupported size or feature";
    case NURSD_ERR_POINT_OUT_OF_RANGE: return "relay sample outside the aperture";
    default: return "unknown status";
  }
}

int nursd_phasor_frequencies(double lambda_c, double dt, int32_t t_pad, int32_t F, double* h_omega, double* h_weight) {
  if (!(lambda_c > 0) || !(dt > 0) || t_pad <= 0 || F <= 0 || !h_omega || !h_weight) return NURSD_ERR_INVALID_ARG;
  const double f_c = kC / lambda_c;
  const double f0 = std::floor(f_c * t_pad * dt + 0.5) - (double)(F / 2);
  const double w_c = 2.0 * kPi * f_c, sigma = w_c / 5.0;
  for (int f = 0; f < F; ++f) {
    const double w = 2.0 * kPi * (f0 + f) / ((double)t_pad * dt);
    h_omega[f] = w;
    h_weight[f] = std::exp(-(w - w_c) * (w - w_c) / (2.0 * sigma * sigma));
  }
  return NURSD_OK;
}

int nursd_subsample(int32_t N, int32_t F, int32_t D, const nursd_c64* d_full, nursd_c64* d_kept,
                    nursd_stream_t stream) {
  if (N < 1 || F < 1 || D < 1 || D > N || !d_full || !d_kept || !aligned(d_full, 8) || !aligned(d_kept, 8))
    return NURSD_ERR_INVALID_ARG;
  return from_cuda(launch_subsample(reinterpret_cast<const float2*>(d_full), reinterpret_cast<float2*>(d_kept), N, F,
                                    D, static_cast<cudaStream_t>(stream)));
}

int nursd_upsample(int32_t N, int32_t F, int32_t D, int32_t mode, const nursd_c64* d_kept, nursd_c64* d_full,
                   nursd_stream_t stream) {
  if (N < 1 || F < 1 || D < 1 || D > N || !d_full || !d_kept || !aligned(d_full, 8) || !aligned(d_kept, 8) ||
      (mode != NURSD_UPSAMPLE_NEAREST && mode != NURSD_UPSAMPLE_LINEAR))
    return NURSD_ERR_INVALID_ARG;
  return from_cuda(launch_upsample(reinterpret_cast<const float2*>(d_kept), reinterpret_cast<float2*>(d_full), N, F,
                                   D, mode == NURSD_UPSAMPLE_LINEAR ? 1 : 0, static_cast<cudaStream_t>(stream)));
}

int nursd_plan_create(const nursd_desc* d, nursd_stream_t stream, nursd_plan_t* out) {
  if (!out) return NURSD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d) return NURSD_ERR_INVALID_ARG;
  if (!is_pow2(d->N) || d->N < 8 || d->N > 512) return NURSD_ERR_UNSUPPORTED;
  if (!(d->pitch > 0) || !std::isfinite(d->pitch) || !std::isfinite(d->center_x) || !std::isfinite(d->center_y))
    return NURSD_ERR_INVALID_ARG;
  if (d->Z < 1 || d->Z > 4096 || !d->h_depths || d->F < 1 || d->F > 256 || !d->h_omega) return NURSD_ERR_INVALID_ARG;
  for (int i = 0; i < d->Z; ++i)
    if (!(d->h_depths[i] > 0) || !std::isfinite(d->h_depths[i])) return NURSD_ERR_INVALID_ARG;
  for (int i = 0; i < d->F; ++i) {
    if (!std::isfinite(d->h_omega[i]) || d->h_omega[i] < 0) return NURSD_ERR_INVALID_ARG;
    if (d->h_weight && !std::isfinite(d->h_weight[i])) return NURSD_ERR_INVALID_ARG;
  }
  if (!std::isfinite(d->lambda_c) || d->lambda_c < 0) return NURSD_ERR_INVALID_ARG;
  if (d->T < 0 || (d->T > 0 && (d->T % 8 != 0 || !(d->dt > 0) || !std::isfinite(d->t0)))) return NURSD_ERR_INVALID_ARG;
  if (d->upsample != 2) return NURSD_ERR_UNSUPPORTED;
  if (d->kernel_width < 4 || d->kernel_width > kMaxKernelWidth) return NURSD_ERR_UNSUPPORTED;
  if (d->max_points < 0 || d->max_points > (1 << 26)) return NURSD_ERR_INVALID_ARG;
  if (d->max_batch < 0 || d->max_batch > kMaxBatch) return NURSD_ERR_INVALID_ARG;
  if (d->max_batch > 0 && d->T <= 0) return NURSD_ERR_INVALID_ARG;
  if (d->h_srsd_pitch)
    for (int i = 0; i < d->Z; ++i)
      if (!(d->h_srsd_pitch[i] > 0) || !std::isfinite(d->h_srsd_pitch[i])) return NURSD_ERR_INVALID_ARG;
  if ((d->flags & ~(NURSD_OUTPUT_MAGNITUDE | NURSD_ENABLE_ADJOINT | NURSD_CONFOCAL)) != 0) return NURSD_ERR_UNSUPPORTED;
  if ((d->flags & NURSD_ENABLE_ADJOINT) && d->Z > 256) return NURSD_ERR_UNSUPPORTED;

  nursd_plan_s* p = new (std::nothrow) nursd_plan_s();
  if (!p) return NURSD_ERR_OOM;
  cudaGetDevice(&p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  p->N = d->N;
  p->M = 2 * d->N;
  p->nf = d->upsample * p->M;
  p->Z = d->Z;
  p->F = d->F;
  p->T = d->T;
  p->w = d->kernel_width;
  p->pitch = d->pitch;
  p->cx = d->center_x;
  p->cy = d->center_y;
  p->t0 = d->t0;
  p->dt = d->dt;
  p->flags = d->flags;
  p->maxL = d->max_points;
  p->maxB = d->max_batch;
  p->beta = (float)(2.30 * p->w);
  p->depths.assign(d->h_depths, d->h_depths + d->Z);
  p->omega.assign(d->h_omega, d->h_omega + d->F);
  p->weight.assign(d->F, 1.0);
  if (!d->h_weight && d->lambda_c > 0) {  // the band-pass of Eq. PFPacket (sigma_w = w_c / 5)
    const double w_c = 2.0 * kPi * kC / d->lambda_c, sigma = w_c / 5.0;
    for (int f = 0; f < d->F; ++f) {
      const double dw = d->h_omega[f] - w_c;
      p->weight[f] = std::exp(-dw * dw / (2.0 * sigma * sigma));
    }
  }
  if (d->h_srsd_pitch) p->srsd_pitch.assign(d->h_srsd_pitch, d->h_srsd_pitch + d->Z);
  if (d->h_weight) p->weight.assign(d->h_weight, d->h_weight + d->F);
  // fine-grid window: every footprint of a sample with |x - c| <= N delta / 2, plus a margin
  const int need = d->upsample * p->N + p->w + 2;
  p->W = (need + kTile - 1) / kTile * kTile;
  p->tiles = p->W / kTile;
  p->g0 = -p->W / 2;
  if (p->W > p->nf) {
    delete p;
    return NURSD_ERR_UNSUPPORTED;
  }
  const int half = p->M / 2;
  p->ncls = (half + 1) * (half + 2) / 2;

  // ---- host tables
  std::vector<float2> tw(kTwiddleEntries);
  for (int e = 0; e < kTwiddleEntries; ++e) {
    int num = 0, lg = 0;
    twiddle_exponent(e, &num, &lg);
    const double a = -2.0 * kPi * num / (double)(1 << lg);
    tw[e] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  std::vector<double> gx, gw;
  gauss_legendre(256, gx, gw);
  std::vector<float> dec(p->M);
  for (int i = 0; i < p->M; ++i) {
    const double k = i - half;
    double s_ = 0.0;
    for (size_t j = 0; j < gx.size(); ++j)
      s_ += gw[j] * es_kernel(gx[j], p->beta) * std::cos(kPi * k * p->w * gx[j] / p->nf);
    dec[i] = (float)(1.0 / (0.5 * p->w * s_));
  }
  std::vector<int2> cls;
  cls.reserve(p->ncls);
  for (int pp = 0; pp <= half; ++pp)
    for (int qq = 0; qq <= pp; ++qq) cls.push_back(make_int2(pp, qq));
  // temporal twiddles, transposed: B^T[2f][n] = cos(w_f t_n), B^T[2f+1][n] = -sin(w_f t_n)
  // (FP64, phase reduced mod 2 pi), stored as fp16 head + tail for the tensor-core GEMM; the
  // weight w_f multiplies the accumulator (column weights wc), so no weight is rounded to fp16
  std::vector<__half> Bth, Btl;
  std::vector<float> wc(2 * (size_t)p->F);
  for (int f = 0; f < p->F; ++f) wc[2 * f] = wc[2 * f + 1] = (float)p->weight[f];
  if (p->T > 0) {
    Bth.resize((size_t)p->T * 2 * p->F);
    Btl.resize(Bth.size());
    for (int f = 0; f < p->F; ++f)
      for (int n = 0; n < p->T; ++n) {
        const double ph = std::fmod(p->omega[f] * (p->t0 + n * p->dt), 2.0 * kPi);
        const double v[2] = {std::cos(ph), -std::sin(ph)};
        for (int c = 0; c < 2; ++c) {
          const __half hi = __float2half_rn((float)v[c]);
          const size_t idx = (size_t)(2 * f + c) * p->T + n;
          Bth[idx] = hi;
          Btl[idx] = __float2half_rn((float)(v[c] - (double)__half2float(hi)));
        }
      }
  }

  // ---- device memory
  const int maxL = std::max(1, p->maxL);
  const int nbins = points_bins(p->W, p->tiles);
  bool ok = p->alloc(p->twiddle, tw.size()) && p->alloc(p->deconv, p->M) && p->alloc(p->cls, p->ncls) &&
            p->alloc(p->Gc, (size_t)p->ncls * p->F * p->Z) && p->alloc(p->status, 1) &&
            p->alloc(p->bin_of, maxL) && p->alloc(p->i0_orig, maxL) && p->alloc(p->w_orig, (size_t)maxL * 2 * p->w) &&
            p->alloc(p->counts, (size_t)2 * nbins) && p->alloc(p->bin_start, nbins + 1) &&
            p->alloc(p->sorted_l, maxL) && p->alloc(p->slot_of, maxL) && p->alloc(p->i0_sorted, maxL) &&
            p->alloc(p->w_sorted, (size_t)maxL * 2 * p->w) && p->alloc(p->phasor, (size_t)maxL * p->F) &&
            p->alloc(p->frac_orig, maxL) && p->alloc(p->frac_sorted, maxL) &&
            p->alloc(p->fine, (size_t)p->W * p->W * std::max(p->F, p->Z)) &&
            p->alloc(p->R1, (size_t)p->W * p->M * std::max(p->F, p->Z)) &&
            p->alloc(p->U, (size_t)p->M * p->M * p->F) && p->alloc(p->Y, (size_t)p->M * p->M * p->Z) &&
            p->alloc(p->T1, (size_t)p->M * p->N * p->Z);
  if (ok && p->T > 0) {  // the row list holds every row a call can pass: maxL, or maxB items of maxL
    const size_t rows = (size_t)maxL * std::max(1, p->maxB);
    ok = p->alloc(p->Bth, Bth.size()) && p->alloc(p->Btl, Btl.size()) && p->alloc(p->wcol, wc.size()) &&
         p->alloc(p->tfix.count, 2) && p->alloc(p->tfix.list, rows);
    if (ok) p->tfix.done = p->tfix.count + 1;
    p->tfix.cap = (int)std::min<size_t>(rows, 1u << 30);
  }
  if (ok && (p->flags & NURSD_ENABLE_ADJOINT))
    ok = p->alloc(p->GcT, (size_t)p->ncls * p->F * p->Z) && p->alloc(p->deconv_k, p->M) &&
         p->alloc(p->fine_dx, (size_t)p->W * p->W * p->F) && p->alloc(p->fine_dy, (size_t)p->W * p->W * p->F);
  if (ok && p->maxB > 0) {  // the batched form's item workspaces, as many items as fit in 8 GiB
    auto& g = p->gst;
    const size_t C = std::max(p->F, p->Z);
    g.pts = maxL;
    g.wts = (size_t)maxL * 2 * p->w;
    g.counts = (size_t)2 * nbins;
    g.bins = (size_t)nbins + 1;
    g.fine = (size_t)p->W * p->W * C;
    g.R1 = (size_t)p->W * p->M * C;
    g.T1 = (size_t)p->M * p->N * p->Z;
    const size_t per_item = g.pts * (3 * sizeof(int) + 4 * sizeof(int2)) + g.wts * 2 * sizeof(float) +
                            (g.counts + g.bins) * sizeof(int) + (g.fine + g.R1 + g.T1) * sizeof(float2);
    const size_t budget = size_t(8) << 30;
    p->group = (int)std::min<size_t>(p->maxB, std::max<size_t>(1, budget / per_item));
    p->group_size = p->group;
    const size_t G = p->group;
    Workspace& w = p->gws;
    ok = p->alloc(w.bin_of, G * g.pts) && p->alloc(w.i0_orig, G * g.pts) && p->alloc(w.w_orig, G * g.wts) &&
         p->alloc(w.counts, G * g.counts) && p->alloc(w.bin_start, G * g.bins) && p->alloc(w.sorted_l, G * g.pts) &&
         p->alloc(w.slot_of, G * g.pts) && p->alloc(w.i0_sorted, G * g.pts) && p->alloc(w.w_sorted, G * g.wts) &&
         p->alloc(w.frac_orig, G * g.pts) && p->alloc(w.frac_sorted, G * g.pts) && p->alloc(w.fine, G * g.fine) &&
         p->alloc(w.R1, G * g.R1) && p->alloc(w.T1, G * g.T1);
    if (ok) ok = cudaMemsetAsync(w.bin_start, 0, sizeof(int) * G * g.bins, s) == cudaSuccess;
  }
  for (int k = 1; ok && p->maxB > 0 && k < kMaxBatchStreams; ++k) {  // the per-item form's other streams
    if (cudaStreamCreateWithFlags(&p->bstream[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->bev_join[k], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  }
  if (ok && p->maxB > 0 && cudaEventCreateWithFlags(&p->bev_fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ok = false;
  }
  if (ok && p->maxB > 0)
    ok = p->alloc(p->phasor_all, (size_t)p->maxB * maxL * p->F) &&
         p->alloc(p->U_all, (size_t)p->maxB * p->M * p->M * p->F) &&
         p->alloc(p->Y_all, (size_t)p->maxB * p->M * p->M * p->Z) && p->alloc(p->counter, 1);
  if (ok && !p->srsd_pitch.empty()) ok = alloc_srsd(p) == NURSD_OK;
  if (!ok) {
    delete p;
    return NURSD_ERR_OOM;
  }
  int rc = from_cuda(cudaMemcpyAsync(p->twiddle, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK)
    rc = from_cuda(cudaMemcpyAsync(p->deconv, dec.data(), sizeof(float) * dec.size(), cudaMemcpyHostToDevice, s));
  std::vector<float> deck(p->M);
  for (int i = 0; i < p->M; ++i) deck[i] = (float)((i - half) * (double)dec[i]);
  if (rc == NURSD_OK && p->deconv_k)
    rc = from_cuda(cudaMemcpyAsync(p->deconv_k, deck.data(), sizeof(float) * deck.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK)
    rc = from_cuda(cudaMemcpyAsync(p->cls, cls.data(), sizeof(int2) * cls.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK && p->T > 0)
    rc = from_cuda(cudaMemcpyAsync(p->Bth, Bth.data(), sizeof(__half) * Bth.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK && p->T > 0)
    rc = from_cuda(cudaMemcpyAsync(p->Btl, Btl.data(), sizeof(__half) * Btl.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK && p->T > 0)
    rc = from_cuda(cudaMemcpyAsync(p->wcol, wc.data(), sizeof(float) * wc.size(), cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK && p->T > 0) rc = from_cuda(cudaMemsetAsync(p->tfix.count, 0, 2 * sizeof(int), s));
  if (rc == NURSD_OK) rc = from_cuda(cudaMemsetAsync(p->status, 0, sizeof(int), s));
  if (rc == NURSD_OK) rc = from_cuda(cudaMemsetAsync(p->bin_start, 0, sizeof(int) * (nbins + 1), s));
  if (rc == NURSD_OK && p->T > 0) make_temporal_maps(p->Bth, p->Btl, p->T, 2 * p->F, &p->tmaps);
  if (rc == NURSD_OK) rc = build_table(p, false, s);
  if (rc == NURSD_OK && p->Gs) rc = build_table(p, true, s);
  if (rc == NURSD_OK && p->Gs) rc = build_srsd_chirps(p, s);
  if (rc != NURSD_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return NURSD_OK;
}

int nursd_plan(const nursd_desc* desc, nursd_stream_t stream, nursd_plan_t* out) {
  return nursd_plan_create(desc, stream, out);
}

int nursd_plan_destroy(nursd_plan_t plan) {
  delete plan;
  return NURSD_OK;
}

int64_t nursd_plan_bytes(nursd_plan_t plan) { return plan ? plan->bytes : -1; }

int nursd_plan_dims(nursd_plan_t plan, int32_t* M, int32_t* fine_n, int32_t* n_classes) {
  if (!plan) return NURSD_ERR_INVALID_ARG;
  if (M) *M = plan->M;
  if (fine_n) *fine_n = plan->nf;
  if (n_classes) *n_classes = plan->ncls;
  return NURSD_OK;
}

namespace {
// Coordinate map, weights and bin sort of L samples on stream s (Sec. 6, NUFFT-1 step 1).
PointsArgs points_args(const nursd_plan_s* p, int32_t L, const float* d_xy) {
  PointsArgs a;
  a.xy = d_xy;
  a.L = L;
  a.cx = p->cx;
  a.cy = p->cy;
  a.inv_fine_pitch = 2.0 / p->pitch;  // sigma / delta
  a.half_extent = 0.5 * p->N * p->pitch;
  a.g0 = p->g0;
  a.W = p->W;
  a.tiles = p->tiles;
  a.width = p->w;
  a.beta = p->beta;
  a.status = p->status;
  return a;
}

int set_points_on(nursd_plan_t p, int32_t L, const float* d_xy, cudaStream_t s) {
  const PointsArgs a = points_args(p, L, d_xy);
  int rc;
  {
    StageTimer t(p, NURSD_STAGE_POINTS, s, L > 0 ? 5 : 0);
    rc = from_cuda(launch_points(a, p->bin_of, p->i0_orig, p->w_orig, p->counts, p->bin_start, p->sorted_l,
                                 p->i0_sorted, p->w_sorted, s, p->frac_orig, p->frac_sorted, p->slot_of));
  }
  if (rc == NURSD_OK) p->L = L;
  return rc;
}
}  // namespace

int nursd_set_points(nursd_plan_t p, int32_t L, const float* d_xy, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || L < 0 || L > p->maxL || (L > 0 && (!d_xy || !aligned(d_xy, 8))))
    return NURSD_ERR_INVALID_ARG;
  p->nd_points = false;
  return set_points_on(p, L, d_xy, static_cast<cudaStream_t>(stream));
}

int nursd_temporal_dft(nursd_plan_t p, int32_t L, const float* d_hist, nursd_c64* d_phasor, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || p->T <= 0 || L < 0 || L > p->maxL) return NURSD_ERR_INVALID_ARG;
  if (L > 0 && (!d_hist || !d_phasor || !aligned(d_hist, 16) || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  StageTimer t(p, NURSD_STAGE_TEMPORAL, static_cast<cudaStream_t>(stream), L > 0 ? kTemporalLaunches : 0);
  return from_cuda(run_temporal(p, d_hist, reinterpret_cast<float*>(d_phasor), L, static_cast<cudaStream_t>(stream)));
}

int nursd_nufft1(nursd_plan_t p, const nursd_c64* d_phasor, nursd_c64* d_spectrum, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || p->L < 0 || !d_spectrum || !aligned(d_spectrum, 8)) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  return run_nufft1(p, reinterpret_cast<const float2*>(d_phasor), reinterpret_cast<float2*>(d_spectrum),
                    static_cast<cudaStream_t>(stream));
}

int nursd_propagate(nursd_plan_t p, const nursd_c64* d_spectrum, void* d_out, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !d_spectrum || !d_out || !aligned(d_spectrum, 8) || !aligned(d_out, 8))
    return NURSD_ERR_INVALID_ARG;
  return run_propagate(p, reinterpret_cast<const float2*>(d_spectrum), d_out, static_cast<cudaStream_t>(stream));
}

int nursd_forward_phasor(nursd_plan_t p, const nursd_c64* d_phasor, void* d_out, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || p->L < 0 || !d_out || !aligned(d_out, 8)) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = run_nufft1(p, reinterpret_cast<const float2*>(d_phasor), p->U, s);
  if (rc == NURSD_OK) rc = run_propagate(p, p->U, d_out, s);
  return rc;
}

int nursd_forward(nursd_plan_t p, const float* d_hist, void* d_out, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || p->T <= 0 || p->L < 0 || !d_out || !aligned(d_out, 8)) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_hist || !aligned(d_hist, 16))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc;
  {
    StageTimer t(p, NURSD_STAGE_TEMPORAL, s, p->L > 0 ? kTemporalLaunches : 0);
    // phasors straight into the spread's sorted order (the internal buffer is read only by the spread)
    rc = from_cuda(run_temporal(p, d_hist, reinterpret_cast<float*>(p->phasor), p->L, s, p->slot_of));
  }
  if (rc == NURSD_OK) rc = run_nufft1(p, p->phasor, p->U, s, true);
  if (rc == NURSD_OK) rc = run_propagate(p, p->U, d_out, s);
  return rc;
}

int nursd_reconstruct(nursd_plan_t p, int32_t L, const float* d_xy, const float* d_hist, void* d_out,
                      nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || p->T <= 0 || L < 0 || L > p->maxL || !d_out || !aligned(d_out, 8))
    return NURSD_ERR_INVALID_ARG;
  if (L > 0 && (!d_xy || !aligned(d_xy, 8) || !d_hist || !aligned(d_hist, 16))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->side) {
    if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return NURSD_ERR_CUDA;
    }
  }
  // fork: the point sort waits for everything before this call on `stream`, then runs beside
  // the temporal transform; the join orders it before the spread (and so before every later
  // operation on `stream`)
  int rc = from_cuda(cudaEventRecord(p->ev_fork, s));
  if (rc == NURSD_OK) rc = from_cuda(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
  if (rc == NURSD_OK) rc = set_points_on(p, L, d_xy, p->side);
  if (rc == NURSD_OK) rc = from_cuda(cudaEventRecord(p->ev_join, p->side));
  if (rc != NURSD_OK) return rc;
  {
    StageTimer t(p, NURSD_STAGE_TEMPORAL, s, L > 0 ? kTemporalLaunches : 0);
    rc = from_cuda(run_temporal(p, d_hist, reinterpret_cast<float*>(p->phasor), L, s));
  }
  const int rj = from_cuda(cudaStreamWaitEvent(s, p->ev_join, 0));  // join even if the temporal launch failed
  if (rc == NURSD_OK) rc = rj;
  if (rc == NURSD_OK) rc = run_nufft1(p, p->phasor, p->U, s);
  if (rc == NURSD_OK) rc = run_propagate(p, p->U, d_out, s);
  return rc;
}

int nursd_adjoint(nursd_plan_t p, const nursd_c64* d_vol, nursd_c64* d_phasor, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !p->GcT || p->L < 0 || !d_vol || !aligned(d_vol, 8)) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = run_adjoint_spectrum(p, reinterpret_cast<const float2*>(d_vol), s);
  if (rc == NURSD_OK) rc = run_type2_to_fine(p, p->U, p->F, false, 1.f, s);
  if (rc == NURSD_OK) {
    StageTimer t(p, NURSD_STAGE_SPREAD, s, p->L > 0 ? 1 : 0);
    InterpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.fine = p->fine;
    a.W = p->W;
    a.F = p->F;
    a.width = p->w;
    a.L = p->L;
    a.beta = p->beta;
    a.sorted_l = p->sorted_l;
    a.i0 = p->i0_sorted;
    a.wts = p->w_sorted;
    a.scale = 1.f;
    a.out = reinterpret_cast<float2*>(d_phasor);
    rc = from_cuda(launch_interp_points(a, s));
  }
  return rc;
}

int nursd_grad_points(nursd_plan_t p, const nursd_c64* d_w, const nursd_c64* d_phasor, nursd_c64* d_grad_phasor,
                      float* d_grad_xy, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !p->GcT || p->L < 0 || !d_w || !aligned(d_w, 8)) return NURSD_ERR_INVALID_ARG;
  if (!d_grad_phasor && !d_grad_xy) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && d_grad_xy && (!d_phasor || !aligned(d_phasor, 8) || !aligned(d_grad_xy, 8)))
    return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && d_grad_phasor && !aligned(d_grad_phasor, 8)) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = run_adjoint_spectrum(p, reinterpret_cast<const float2*>(d_w), s);
  if (rc == NURSD_OK && d_grad_phasor) rc = run_type2_to_fine(p, p->U, p->F, false, 1.f, s);
  if (rc == NURSD_OK && d_grad_xy) {  // the spectral derivative: type 2 of kx R and of ky R
    rc = run_type2_to_fine(p, p->U, p->F, false, 1.f, s, p->deconv_k, p->deconv, p->fine_dx);
    if (rc == NURSD_OK) rc = run_type2_to_fine(p, p->U, p->F, false, 1.f, s, p->deconv, p->deconv_k, p->fine_dy);
  }
  if (rc == NURSD_OK) {
    StageTimer t(p, NURSD_STAGE_SPREAD, s, p->L > 0 ? 1 : 0);
    InterpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.fine = p->fine;
    a.fine_dx = p->fine_dx;
    a.fine_dy = p->fine_dy;
    a.W = p->W;
    a.F = p->F;
    a.width = p->w;
    a.L = p->L;
    a.beta = p->beta;
    a.dudx = (float)(2.0 * kPi / (p->M * p->pitch));  // d theta / dx
    a.sorted_l = p->sorted_l;
    a.i0 = p->i0_sorted;
    a.wts = p->w_sorted;
    a.scale = 1.f;
    a.out = reinterpret_cast<float2*>(d_grad_phasor);
    a.P = reinterpret_cast<const float2*>(d_phasor);
    a.gxy = d_grad_xy;
    rc = from_cuda(launch_interp_points(a, s));
  }
  return rc;
}

// Type-2 output of the depth spectra in p->Y at K voxels per plane (NURSD-2/3): deconvolve, pad,
// inverse fine-grid transform per plane, ES interpolation.  plane_scale [Z] (device) or null:
// plane z's lattice pitch over the plan's (SRSD's scaled planes).
int run_points_output(nursd_plan_s* p, int K, const float* d_vox_xy, const double* plane_scale, nursd_c64* d_out,
                      cudaStream_t s) {
  const int M = p->M;
  int rc = run_type2_to_fine(p, p->Y, p->Z, true, 1.f / ((float)M * (float)M), s);
  if (rc == NURSD_OK && K > 0) {
    StageTimer t(p, NURSD_STAGE_IFFT_Y, s, 1);
    PlaneInterpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.fine = p->fine;
    a.W = p->W;
    a.Z = p->Z;
    a.K = K;
    a.width = p->w;
    a.g0 = p->g0;
    a.beta = p->beta;
    a.cx = p->cx;
    a.cy = p->cy;
    a.inv_fine_pitch = 2.0 / p->pitch;
    a.half_extent = 0.5 * p->N * p->pitch;
    a.plane_scale = plane_scale;
    a.vox = d_vox_xy;
    a.scale = 1.f;
    a.out = reinterpret_cast<float2*>(d_out);
    a.status = p->status;
    rc = from_cuda(launch_interp_planes(a, s));
  }
  return rc;
}

int nursd_forward_points(nursd_plan_t p, const nursd_c64* d_phasor, int32_t K, const float* d_vox_xy,
                         nursd_c64* d_out, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || p->L < 0 || K < 0) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  if (K > 0 && (!d_vox_xy || !d_out || !aligned(d_vox_xy, 8) || !aligned(d_out, 8))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int M = p->M;
  int rc = run_nufft1(p, reinterpret_cast<const float2*>(d_phasor), p->U, s);
  if (rc == NURSD_OK) {
    StageTimer t(p, NURSD_STAGE_CONTRACT, s, 1);
    rc = from_cuda(contract_forward(p, p->U, s));
  }
  if (rc == NURSD_OK) rc = run_points_output(p, K, d_vox_xy, nullptr, d_out, s);
  return rc;
}

int srsd_forward(nursd_plan_t p, const nursd_c64* d_phasor, void* d_out, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !p->Gs || p->L < 0 || !d_out || !aligned(d_out, 8)) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = run_nufft1(p, reinterpret_cast<const float2*>(d_phasor), p->U, s);
  if (rc == NURSD_OK) rc = run_srsd_spectra(p, s);
  if (rc == NURSD_OK) rc = run_idft_crop(p, d_out, s);
  return rc;
}

int srsd_forward_at(nursd_plan_t p, const double* h_pitch, const nursd_c64* d_phasor, void* d_out,
                    nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !h_pitch) return NURSD_ERR_INVALID_ARG;
  for (int z = 0; z < p->Z; ++z)
    if (!(h_pitch[z] > 0) || !std::isfinite(h_pitch[z])) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->srsd_pitch.size() != (size_t)p->Z || !std::equal(p->srsd_pitch.begin(), p->srsd_pitch.end(), h_pitch)) {
    // new pitches: the tables in use may still be read by work queued on the stream
    if (cudaStreamSynchronize(s) != cudaSuccess) return NURSD_ERR_CUDA;
    p->srsd_pitch.assign(h_pitch, h_pitch + p->Z);
    p->nu_ready = false;  // the NU-SFFT taps follow the scales
    int rc = alloc_srsd(p);
    if (rc == NURSD_OK) rc = build_table(p, true, s);
    if (rc == NURSD_OK) rc = build_srsd_chirps(p, s);
    if (rc == NURSD_OK) rc = from_cuda(cudaStreamSynchronize(s));
    if (rc != NURSD_OK) return rc;
  }
  return srsd_forward(p, d_phasor, d_out, stream);
}

int srsd_forward_points(nursd_plan_t p, const nursd_c64* d_phasor, int32_t K, const float* d_vox_xy, nursd_c64* d_out,
                        nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !p->Gs || p->L < 0 || K < 0) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  if (K > 0 && (!d_vox_xy || !d_out || !aligned(d_vox_xy, 8) || !aligned(d_out, 8))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = run_nufft1(p, reinterpret_cast<const float2*>(d_phasor), p->U, s);
  if (rc == NURSD_OK) rc = run_srsd_spectra(p, s);
  if (rc == NURSD_OK) rc = run_points_output(p, K, d_vox_xy, p->srsd_scale_d, d_out, s);
  return rc;
}

int srsd_forward_nonuniform(nursd_plan_t p, const nursd_c64* d_phasor, void* d_out, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !p->Gs || p->L < 0 || !d_out || !aligned(d_out, 8)) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_nusfft(p, s);
  if (rc == NURSD_OK) rc = run_nusfft_spectra(p, reinterpret_cast<const float2*>(d_phasor), s);
  if (rc == NURSD_OK) rc = run_idft_crop(p, d_out, s);
  return rc;
}

int nursd_enable_3d(nursd_plan_t p, double dz, int32_t Mz, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !(dz > 0) || !std::isfinite(dz)) return NURSD_ERR_INVALID_ARG;
  if (p->nd_Mz) return (Mz == p->nd_Mz && dz == p->nd_dz) ? NURSD_OK : NURSD_ERR_INVALID_ARG;
  // the z window of footprints must fit one period of the 2 Mz fine grid
  if (!is_pow2(Mz) || Mz < 8 || Mz > 512 || Mz < p->w + 2) return NURSD_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int M = p->M, N = p->N, F = p->F, maxL = std::max(1, p->maxL);
  p->nd_Mz = Mz;
  p->nd_dz = dz;
  p->nd_Wz = std::min(2 * Mz, Mz + p->w + 2);
  p->nd_gz0 = -(Mz / 2) - p->w / 2 - 1;
  if (p->nd_Wz == 2 * Mz) p->nd_gz0 = -Mz;
  if (!(p->alloc(p->nd_G3, (size_t)M * M * Mz * F) && p->alloc(p->nd_U3w, (size_t)p->nd_Wz * M * M * F) &&
        p->alloc(p->nd_U3, (size_t)M * M * Mz * F) && p->alloc(p->nd_What, (size_t)M * M * F) &&
        p->alloc(p->nd_field, (size_t)F * N * N) && p->alloc(p->nd_T, (size_t)N * M * F) &&
        p->alloc(p->nd_decz, Mz) && p->alloc(p->nd_uz, maxL))) {
    p->nd_Mz = 0;
    return NURSD_ERR_OOM;
  }
  {  // stage 1 in groups of z slices: each slice's phasors, window and rows, as many slices as 4 GiB hold
    const size_t per_slice = sizeof(float2) * ((size_t)maxL * F + (size_t)p->W * p->W * F + (size_t)p->W * M * F);
    p->nd_G = (int)std::max<size_t>(1, std::min<size_t>(p->nd_Wz, (size_t(4) << 30) / per_slice));
    const size_t G = p->nd_G;
    if (!(p->alloc(p->nd_Pz, G * maxL * F) && p->alloc(p->nd_fine, G * p->W * p->W * F) &&
          p->alloc(p->nd_R1, G * p->W * M * F))) {
      p->nd_Mz = 0;
      return NURSD_ERR_OOM;
    }
  }
  p->nd_host.resize(Mz);
  for (int i = 0; i < Mz; ++i) p->nd_host[i] = (float)(1.0 / es_transform(i - Mz / 2, p->w, p->beta, 2 * Mz));
  int rc = from_cuda(cudaMemcpyAsync(p->nd_decz, p->nd_host.data(), sizeof(float) * Mz, cudaMemcpyHostToDevice, s));
  if (rc == NURSD_OK) rc = build_table_3d(p, s);
  if (rc != NURSD_OK) p->nd_Mz = 0;
  return rc;
}

int nursd_set_points_3d(nursd_plan_t p, int32_t L, const float* d_xy, const float* d_h, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !p->nd_Mz || L < 0 || L > p->maxL) return NURSD_ERR_INVALID_ARG;
  if (L > 0 && (!d_xy || !d_h || !aligned(d_xy, 8) || !aligned(d_h, 4))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = set_points_on(p, L, d_xy, s);
  if (rc == NURSD_OK)  // fine z coordinate h * 2 / dz, |h| <= Mz dz / 4 (theta_z in [-pi/2, pi/2])
    rc = from_cuda(launch_z_coords(d_h, p->sorted_l, L, 2.0 / p->nd_dz, 0.25 * p->nd_Mz * p->nd_dz, p->nd_uz,
                                   p->status, s));
  p->nd_points = rc == NURSD_OK;
  return rc;
}

int nursd_forward_3d(nursd_plan_t p, const nursd_c64* d_phasor, void* d_out, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || !p->nd_Mz || !p->nd_points || p->L < 0 || !d_out || !aligned(d_out, 8))
    return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int M = p->M, N = p->N, F = p->F, W = p->W, Mz = p->nd_Mz, L = p->L;
  const int logf = ilog2(p->nf), logM = ilog2(M);
  const long long MMF = (long long)M * M * F;
  cudaError_t e = cudaSuccess;
  // stage 1, 3D type 1: per fine z cell of the window, the slice's phasors, the planar spread and the
  // lateral passes with deconvolution -> the slice's lateral spectrum; each step one launch over a
  // group of nd_G slices (the slice the outer index of the phasors, windows and rows)
  const long long pz_stride = (long long)std::max(1, p->maxL) * F;
  for (int iz0 = 0; e == cudaSuccess && iz0 < p->nd_Wz; iz0 += p->nd_G) {
    const int n = std::min(p->nd_G, p->nd_Wz - iz0);
    {
      StageTimer t(p, NURSD_STAGE_SPREAD, s, 2);
      e = launch_z_slice_phasors(reinterpret_cast<const float2*>(d_phasor), p->sorted_l, p->nd_uz, L, F,
                                 p->nd_gz0 + iz0, n, pz_stride, p->w, p->beta, p->nd_Pz, s);
      if (e == cudaSuccess) {
        SpreadItems si;  // the same sorted samples for every slice, its own phasors and window
        si.n = n;
        si.p_stride = pz_stride;
        si.fine_stride = (long long)W * W * F;
        si.status = p->status;
        si.uz = p->nd_uz;  // each slice spreads only the samples its z cell reaches
        si.gz_first = p->nd_gz0 + iz0;
        e = launch_spread(p->nd_Pz, F, p->bin_start, nullptr, p->i0_sorted, p->w_sorted, p->w, p->tiles, W,
                          p->nd_fine, s, p->spread_rows, si);
      }
    }
    if (e == cudaSuccess) {  // along x: the windows' rows back to back
      StageTimer t(p, NURSD_STAGE_FFT_X, s, 1);
      e = axis_pass(p, p->nd_fine, p->nd_R1, logf, false, F, n * W, (long long)W * F, F, (long long)M * F, F, W,
                    p->g0, M, -M / 2, nullptr, nullptr, 1.f, s);
    }
    if (e == cudaSuccess) {  // along y with the deconvolution, the slice as the panels' outer channel index
      StageTimer t(p, NURSD_STAGE_FFT_Y, s, 1);
      e = axis_pass(p, p->nd_R1, p->nd_U3w + iz0 * MMF, logf, false, F, M, F, (long long)M * F, F, (long long)M * F,
                    W, p->g0, M, -M / 2, p->deconv, p->deconv, 1.f, s, n, (long long)W * M * F, MMF);
    }
  }
  if (e == cudaSuccess) {  // along z: the window's slices -> kz in I_Mz, divided by psi_hat_z(kz)
    StageTimer t(p, NURSD_STAGE_FFT_Y, s, 1);
    e = axis_pass(p, p->nd_U3w, p->nd_U3, ilog2(2 * Mz), false, F, M * M, F, MMF, (long long)Mz * F, F, p->nd_Wz,
                  p->nd_gz0, Mz, -Mz / 2, p->nd_decz, nullptr, 1.f, s);
  }
  if (e == cudaSuccess) {  // the plane z0: sum over kz of the spectrum times the 3D table, / Mz
    StageTimer t(p, NURSD_STAGE_CONTRACT, s, 1);
    e = launch_kz_sum(p->nd_U3, p->nd_G3, (long long)M * M, Mz, F, 1.f / (float)Mz, p->nd_What, s);
  }
  // the plane's field on the N x N lattice (M^-2 inverse, crop), then its padded DFT: stage 2's input
  if (e == cudaSuccess) e = idft_crop(p, p->nd_What, F, p->nd_T, p->nd_field, false, s);
  if (e == cudaSuccess) {  // DFT along mx of every (f, my) row of the field [F][N][N] -> [N][M][F]
    StageTimer t(p, NURSD_STAGE_IFFT_Y, s, 1);
    PanelArgs a = panel_base(p);
    a.in = p->nd_field;
    a.in_sb = N;
    a.in_si = 1;
    a.in_slo = (long long)N * N;
    a.load_i_fastest = 1;
    a.out = p->nd_T;
    a.out_sb = (long long)M * F;
    a.out_si = F;
    a.out_slo = 1;
    a.nin = N;
    a.in_off = -N / 2;
    a.nout = M;
    a.out_off = -M / 2;
    a.lo_total = F;
    a.CLO = panel_width(logM);
    a.batch = N;
    e = launch_panel_fft(logM, false, a, s);
  }
  if (e == cudaSuccess) {  // DFT along my for every kx -> U [M][M][F]
    StageTimer t(p, NURSD_STAGE_IFFT_X, s, 1);
    e = axis_pass(p, p->nd_T, p->U, logM, false, F, M, F, (long long)M * F, F, (long long)M * F, N, -N / 2, M, -M / 2,
                  nullptr, nullptr, 1.f, s);
  }
  if (e != cudaSuccess) return from_cuda(e);
  // stage 2: the planar operator from z0 to each depth (the plan's depths are the distances from z0)
  return run_propagate(p, p->U, d_out, s);
}

int nursd_forward_illuminated(nursd_plan_t p, const double* h_illum, const nursd_c64* d_phasor, nursd_c64* d_out,
                              nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || p->L < 0 || !h_illum || !d_out || !aligned(d_out, 8)) return NURSD_ERR_INVALID_ARG;
  if (p->flags & NURSD_CONFOCAL) return NURSD_ERR_UNSUPPORTED;  // the illumination point is each relay point
  if (!(std::isfinite(h_illum[0]) && std::isfinite(h_illum[1]) && std::isfinite(h_illum[2])))
    return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_per_frequency(p, s);
  if (rc == NURSD_OK) rc = run_nufft1(p, reinterpret_cast<const float2*>(d_phasor), p->U, s);
  if (rc == NURSD_OK) rc = run_per_frequency(p, h_illum, 0, reinterpret_cast<float2*>(d_out), s);
  return rc;
}

int nursd_transient_frames(nursd_plan_t p, int32_t n_frames, const double* h_times, const nursd_c64* d_phasor,
                           nursd_c64* d_out, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || p->L < 0 || n_frames < 1 || n_frames > 4096 || !h_times || !d_out ||
      !aligned(d_out, 8))
    return NURSD_ERR_INVALID_ARG;
  for (int t = 0; t < n_frames; ++t)
    if (!std::isfinite(h_times[t])) return NURSD_ERR_INVALID_ARG;
  if (p->L > 0 && (!d_phasor || !aligned(d_phasor, 8))) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_per_frequency(p, s);
  if (rc != NURSD_OK) return rc;
  const int F = p->F;
  if (n_frames > p->pf_A_cap) {
    if (!p->alloc(p->pf_A, (size_t)n_frames * F)) return NURSD_ERR_OOM;
    p->pf_A_cap = n_frames;
  }
  // weights exp(+i w_f t) with the phase reduced in FP64 (w_f t reaches ~1e3 rad), rounded to
  // complex64, uploaded from a plan-owned host copy; stream order puts the upload before this
  // call's sums and after an earlier call's.
  p->pf_A_host.resize((size_t)n_frames * F);
  for (int t = 0; t < n_frames; ++t)
    for (int f = 0; f < F; ++f) {
      const double ph = std::fmod(p->omega[f] * h_times[t], 2.0 * kPi);
      p->pf_A_host[(size_t)t * F + f] = make_float2((float)std::cos(ph), (float)std::sin(ph));
    }
  if (cudaMemcpyAsync(p->pf_A, p->pf_A_host.data(), sizeof(float2) * p->pf_A_host.size(), cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return NURSD_ERR_CUDA;
  rc = run_nufft1(p, reinterpret_cast<const float2*>(d_phasor), p->U, s);
  if (rc == NURSD_OK) rc = run_per_frequency(p, nullptr, n_frames, reinterpret_cast<float2*>(d_out), s);
  return rc;
}

namespace {
// The contraction of B items sharing the table: on the tensor cores when the shape allows (a dense
// product per symmetry class once several items share it), else the bulk-copy SIMT kernel.
cudaError_t contract_items(nursd_plan_s* p, long long u_stride, long long y_stride, int B, cudaStream_t s) {
  if (B >= 2 && p->batch_tensor && contract_umma_supported(p->M, p->F, p->Z, B, u_stride, y_stride))
    return launch_contract_umma(p->U_all, u_stride, p->Gc, p->cls, p->ncls, p->M, p->F, p->Z, p->Y_all, y_stride, B,
                                p->status, s);
  return launch_contract_batched(p->U_all, u_stride, p->Gc, p->cls, p->ncls, p->M, p->F, p->Z, p->Y_all, y_stride, B,
                                 s, p->status);
}
}  // namespace

int nursd_forward_batched(nursd_plan_t p, int32_t B, const nursd_batch_item* items, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK || p->maxB <= 0 || B < 1 || B > p->maxB || !items) return NURSD_ERR_INVALID_ARG;
  for (int b = 0; b < B; ++b) {
    const nursd_batch_item& it = items[b];
    if (it.L < 0 || it.L > p->maxL || !it.d_out || !aligned(it.d_out, 8)) return NURSD_ERR_INVALID_ARG;
    if (it.L > 0 && (!it.d_xy || !it.d_hist || !aligned(it.d_xy, 8) || !aligned(it.d_hist, 16)))
      return NURSD_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int M = p->M, F = p->F, Z = p->Z;
  const size_t phasor_stride = (size_t)std::max(1, p->maxL) * F;
  const long long u_stride = (long long)M * M * F, y_stride = (long long)M * M * Z;
  int rc = NURSD_OK;
  {  // temporal transforms of every item: one persistent launch over the ragged tile list
    StageTimer t(p, NURSD_STAGE_TEMPORAL, s, kTemporalLaunches);
    TemporalBatch bt;
    bt.n = B;
    bt.tile_start[0] = 0;
    const int ncol = (2 * F + 127) / 128;
    for (int b = 0; b < B; ++b) {
      bt.A[b] = items[b].d_hist;
      bt.C[b] = reinterpret_cast<float*>(p->phasor_all + b * phasor_stride);
      bt.L[b] = items[b].L;
      bt.tile_start[b + 1] = bt.tile_start[b] + ((items[b].L + 127) / 128) * ncol;
    }
    bool umma = p->tmaps.ok != 0;
    for (int b = 0; umma && b < B; ++b) umma = aligned(items[b].d_hist, 16) && aligned(bt.C[b], 16);
    if (umma) {  // the tcgen05 form over 128-row tiles of every item, then the gather of listed rows
      TemporalBatch bu = bt;
      for (int b = 0; b < B; ++b) bu.tile_start[b + 1] = bu.tile_start[b] + (items[b].L + 127) / 128;
      rc = from_cuda(launch_temporal_umma_batched(p->tmaps, bu, p->wcol, p->T, 2 * F, p->tfix, p->status, s));
      if (rc == NURSD_OK)
        rc = from_cuda(launch_temporal_tc_gather(bu, p->Bth, p->Btl, p->wcol, p->T, 2 * F, p->tfix, s));
    } else {
      rc = from_cuda(launch_temporal_tc_batched(bt, p->Bth, p->Btl, p->wcol, p->T, 2 * F, p->tfix, p->counter, s));
    }
  }
  // Per item: point sort, spread and the forward fine-grid passes (-> U_all[b]), then after the batched
  // contraction the inverse passes; items go round-robin to S streams (the caller's stream with the
  // plan's own workspace, and up to kMaxBatchStreams - 1 side streams with their own), forked from and
  // joined into the caller's stream, so that the items' small launches run side by side.  The last
  // item runs on the plan's own workspace, so the plan keeps its points as a single call would.
  const int S = std::max(1, std::min(std::min(p->batch_streams, B), p->group));
  const Workspace own = p->own();
  auto fork = [&]() -> int {
    int r = from_cuda(cudaEventRecord(p->bev_fork, s));
    for (int k = 1; r == NURSD_OK && k < S; ++k) r = from_cuda(cudaStreamWaitEvent(p->bstream[k], p->bev_fork, 0));
    return r;
  };
  auto join = [&]() -> int {
    int r = NURSD_OK;
    for (int k = 1; k < S; ++k) {  // join every stream that was forked, even after an error
      const int a = from_cuda(cudaEventRecord(p->bev_join[k], p->bstream[k]));
      const int b = from_cuda(cudaStreamWaitEvent(s, p->bev_join[k], 0));
      if (r == NURSD_OK) r = a != NURSD_OK ? a : b;
    }
    return r;
  };
  auto each_item = [&](auto&& fn) -> int {
    int r = fork();
    for (int b = 0; r == NURSD_OK && b < B; ++b) {
      const int k = (B - 1 - b) % S;
      cudaStream_t sk = k == 0 ? s : p->bstream[k];
      p->use(k == 0 ? own : p->group_item(k));
      r = fn(b, sk);
      p->use(own);
    }
    const int j = join();
    return r != NURSD_OK ? r : j;
  };
  // Grouped form: when the outputs lie side by side (one stride apart) and the plan has it enabled,
  // every stage runs as one launch over a group of up to p->group items (the item index a grid or
  // panel dimension): point sort, spread, both forward passes; then the contraction over all items;
  // then both inverse passes.  The launch count depends on ceil(B / group), not on B.
  const bool mag = (p->flags & NURSD_OUTPUT_MAGNITUDE) != 0;
  const long long ebytes = mag ? (long long)sizeof(float) : (long long)sizeof(float2);
  const long long vol_bytes = (long long)p->N * p->N * Z * ebytes;
  long long out_step = 0;  // elements between consecutive items' outputs
  bool side_by_side = p->batch_grouped != 0 && p->group > 0;
  if (side_by_side && B > 1) {
    const long long d = static_cast<const char*>(items[1].d_out) - static_cast<const char*>(items[0].d_out);
    side_by_side = d >= vol_bytes && d % ebytes == 0;
    for (int b = 2; side_by_side && b < B; ++b)
      side_by_side = static_cast<const char*>(items[b].d_out) - static_cast<const char*>(items[0].d_out) == b * d;
    out_step = d / ebytes;
  }
  if (rc == NURSD_OK && side_by_side) {
    const int N = p->N, W = p->W, G = std::max(1, std::min(p->group_size, p->group));
    const int logf = ilog2(p->nf), logM = ilog2(M);
    const nursd_plan_s::ItemStrides& g = p->gst;
    const Workspace& gw = p->gws;
    const long long fine_st = (long long)W * W * F, r1_st = (long long)W * M * F, t1_st = (long long)M * N * Z;
    // the plan keeps the last item's points, as a single call would: sorted on stream 1 beside the batch
    rc = from_cuda(cudaEventRecord(p->bev_fork, s));
    if (rc == NURSD_OK) rc = from_cuda(cudaStreamWaitEvent(p->bstream[1], p->bev_fork, 0));
    if (rc == NURSD_OK) rc = set_points_on(p, items[B - 1].L, items[B - 1].d_xy, p->bstream[1]);
    const int rj = from_cuda(cudaEventRecord(p->bev_join[1], p->bstream[1]));
    if (rc == NURSD_OK) rc = rj;
    const PointsArgs pa = points_args(p, 0, nullptr);
    for (int g0 = 0; rc == NURSD_OK && g0 < B; g0 += G) {
      const int n = std::min(G, B - g0);
      PointsItems it;
      for (int b = 0; b < n; ++b) {
        it.L[b] = items[g0 + b].L;
        it.xy[b] = items[g0 + b].d_xy;
      }
      {
        StageTimer t(p, NURSD_STAGE_POINTS, s, 5);
        rc = from_cuda(launch_points_batched(pa, it, n, (long long)g.pts, gw.bin_of, gw.i0_orig, gw.w_orig, gw.counts,
                                             gw.bin_start, gw.sorted_l, gw.i0_sorted, gw.w_sorted, nullptr, nullptr,
                                             nullptr, s));
      }
      if (rc == NURSD_OK) {
        StageTimer t(p, NURSD_STAGE_SPREAD, s, 1);
        SpreadItems si;
        si.n = n;
        si.p_stride = (long long)phasor_stride;
        si.pts = (long long)g.pts;
        si.fine_stride = fine_st;
        si.bstride = (int)g.bins;
        si.status = p->status;
        rc = from_cuda(launch_spread(p->phasor_all + g0 * phasor_stride, F, gw.bin_start, gw.sorted_l, gw.i0_sorted,
                                     gw.w_sorted, p->w, p->tiles, W, gw.fine, s, p->spread_rows, si));
      }
      if (rc == NURSD_OK) {  // FFT along x of every window row of every item (rows of items back to back)
        StageTimer t(p, NURSD_STAGE_FFT_X, s, 1);
        rc = from_cuda(axis_pass(p, gw.fine, gw.R1, logf, false, F, n * W, (long long)W * F, F, (long long)M * F, F,
                                 W, p->g0, M, -M / 2, nullptr, nullptr, 1.f, s));
      }
      if (rc == NURSD_OK) {  // FFT along y of every kx column with the deconvolution, items as outer channels
        StageTimer t(p, NURSD_STAGE_FFT_Y, s, 1);
        rc = from_cuda(axis_pass(p, gw.R1, p->U_all + g0 * u_stride, logf, false, F, M, F, (long long)M * F, F,
                                 (long long)M * F, W, p->g0, M, -M / 2, p->deconv, p->deconv, 1.f, s, n, r1_st,
                                 u_stride));
      }
    }
    if (rc == NURSD_OK) {
      StageTimer t(p, NURSD_STAGE_CONTRACT, s, 1);
      rc = from_cuda(contract_items(p, u_stride, y_stride, B, s));
    }
    for (int g0 = 0; rc == NURSD_OK && g0 < B; g0 += G) {
      const int n = std::min(G, B - g0);
      {  // inverse along kx of every ky row of every item, keep mx in I_N
        StageTimer t(p, NURSD_STAGE_IFFT_X, s, 1);
        rc = from_cuda(axis_pass(p, p->Y_all + g0 * y_stride, gw.T1, logM, true, Z, n * M, (long long)M * Z, Z,
                                 (long long)N * Z, Z, M, -M / 2, N, -N / 2, nullptr, nullptr, 1.f, s));
      }
      if (rc == NURSD_OK) {
        char* out0 = static_cast<char*>(items[g0].d_out);
        rc = from_cuda(idft_crop_y(p, gw.T1, Z, out0, mag, s, n, t1_st, out_step));
      }
    }
    const int rw = from_cuda(cudaStreamWaitEvent(s, p->bev_join[1], 0));  // join even after an error
    if (rc == NURSD_OK) rc = rw;
    if (rc == NURSD_OK) p->L = items[B - 1].L;
    return rc;
  }
  if (rc == NURSD_OK)
    rc = each_item([&](int b, cudaStream_t sk) {
      int r = set_points_on(p, items[b].L, items[b].d_xy, sk);
      if (r == NURSD_OK) r = run_nufft1(p, p->phasor_all + b * phasor_stride, p->U_all + b * u_stride, sk);
      return r;
    });
  if (rc == NURSD_OK) {
    StageTimer t(p, NURSD_STAGE_CONTRACT, s, 1);
    rc = from_cuda(contract_items(p, u_stride, y_stride, B, s));
  }
  if (rc == NURSD_OK)
    rc = each_item([&](int b, cudaStream_t sk) { return run_idft_crop(p, items[b].d_out, sk, p->Y_all + b * y_stride); });
  if (rc == NURSD_OK) p->L = items[B - 1].L;
  return rc;
}

int nursd_plan_tune(nursd_plan_t p, int32_t param, int32_t value) {
  if (check_plan(p) != NURSD_OK) return NURSD_ERR_INVALID_ARG;
  switch (param) {
    case NURSD_TUNE_SPREAD_ROWS:
      if (!spread_rows_supported(value) || p->W % value != 0) return NURSD_ERR_UNSUPPORTED;
      p->spread_rows = value;
      return NURSD_OK;
    case NURSD_TUNE_BATCH_STREAMS:
      if (value < 1 || value > kMaxBatchStreams) return NURSD_ERR_UNSUPPORTED;
      p->batch_streams = value;
      return NURSD_OK;
    case NURSD_TUNE_BATCH_GROUPED:
      if (value != 0 && value != 1) return NURSD_ERR_UNSUPPORTED;
      p->batch_grouped = value;
      return NURSD_OK;
    case NURSD_TUNE_BATCH_GROUP:
      if (value < 1 || value > p->group) return NURSD_ERR_UNSUPPORTED;
      p->group_size = value;
      return NURSD_OK;
    case NURSD_TUNE_BATCH_TENSOR:
      if (value != 0 && value != 1) return NURSD_ERR_UNSUPPORTED;
      p->batch_tensor = value;
      return NURSD_OK;
    case NURSD_TUNE_CONTRACT_TC:
      if (value != 0 && value != 1) return NURSD_ERR_UNSUPPORTED;
      p->contract_tc = value;
      return NURSD_OK;
    default:
      return NURSD_ERR_INVALID_ARG;
  }
}

int nursd_plan_get_tune(nursd_plan_t p, int32_t param, int32_t* value) {
  if (check_plan(p) != NURSD_OK || !value) return NURSD_ERR_INVALID_ARG;
  switch (param) {
    case NURSD_TUNE_SPREAD_ROWS: *value = p->spread_rows; return NURSD_OK;
    case NURSD_TUNE_BATCH_STREAMS: *value = p->batch_streams; return NURSD_OK;
    case NURSD_TUNE_BATCH_GROUPED: *value = p->batch_grouped; return NURSD_OK;
    case NURSD_TUNE_BATCH_GROUP: *value = p->group_size; return NURSD_OK;
    case NURSD_TUNE_BATCH_TENSOR: *value = p->batch_tensor; return NURSD_OK;
    case NURSD_TUNE_CONTRACT_TC: *value = p->contract_tc; return NURSD_OK;
    default: return NURSD_ERR_INVALID_ARG;
  }
}

int nursd_test_fail_allocation(int32_t after) {
  g_alloc_countdown.store(after > 0 ? after : -1);
  return NURSD_OK;
}

int nursd_test_set_wait_limit(int64_t polls, nursd_stream_t stream) {
  return from_cuda(set_contract_wait_limit(polls, static_cast<cudaStream_t>(stream)));
}

int nursd_profile_enable(nursd_plan_t p, int enable) {
  return nursd_profile_select(p, enable ? (1u << NURSD_NUM_STAGES) - 1u : 0u);
}

int nursd_profile_select(nursd_plan_t p, uint32_t stage_mask) {
  if (check_plan(p) != NURSD_OK) return NURSD_ERR_INVALID_ARG;
  p->profile_mask = stage_mask & ((1u << NURSD_NUM_STAGES) - 1u);
  p->profiling = p->profile_mask != 0;
  for (auto& u : p->ev_used) u = 0;
  return NURSD_OK;
}

int nursd_profile_read(nursd_plan_t p, int stage, double* h_ms, int64_t* h_count) {
  if (check_plan(p) != NURSD_OK || stage < 0 || stage >= NURSD_NUM_STAGES || !h_ms || !h_count)
    return NURSD_ERR_INVALID_ARG;
  double total = 0.0;
  for (size_t i = 0; i < p->ev_used[stage]; ++i) {
    auto& e = p->ev[stage][i];
    if (cudaEventSynchronize(e.second) != cudaSuccess) return NURSD_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.first, e.second) != cudaSuccess) return NURSD_ERR_CUDA;
    total += ms;
  }
  *h_ms = total;
  *h_count = (int64_t)p->ev_used[stage];
  p->ev_used[stage] = 0;
  return NURSD_OK;
}

int64_t nursd_launch_count(nursd_plan_t p) { return p ? p->launches : -1; }

int nursd_sync_status(nursd_plan_t p, nursd_stream_t stream) {
  if (check_plan(p) != NURSD_OK) return NURSD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  if (cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return NURSD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return NURSD_ERR_CUDA;
  if (h != 0 && cudaMemsetAsync(p->status, 0, sizeof(int), s) != cudaSuccess) return NURSD_ERR_CUDA;
  if (h & 6) return NURSD_ERR_TIMEOUT;  // a bounded barrier wait gave up (contraction, SRSD: 2, temporal: 4)
  if (h & 8) return NURSD_ERR_UNSUPPORTED;  // an SRSD tap table broke the interpolation's step rule
  if (h & 16) return NURSD_ERR_CUDA;  // checked build: an internal index check failed
  if (h & 1) return NURSD_ERR_POINT_OUT_OF_RANGE;
  return NURSD_OK;
}

}  // extern "C"
