/*
 * libnursd -- GB300 (sm_103a) implementation of the non-uniform
 * Rayleigh-Sommerfeld diffraction (NURSD) operator of "Optimized Sampling for
 * Non-Line-of-Sight Imaging Using Modified Fast Fourier Transforms"
 * (arXiv 2501.05244).
 *
 * The operator back-propagates a phasor field measured at an unordered list of
 * relay-wall samples (x_l, y_l) (Sec. 6) into N x N voxel planes at depths z_v:
 *
 *   P[l][f]  = w_f sum_n h_l[n] exp(-i w_f (t0 + n dt))          Eq. PF_Response, PFPacket
 *   U_f(k)   = sum_l P[l][f] exp(-i k . theta_l)                 NUFFT-1 (Sec. 6)
 *   Y_z(k)   = sum_f U_f(k) Ghat_{z,f}(k)                        Eq. 4 product + frequency sum (Eq. 2)
 *   V_z[m]   = M^-2 sum_k Y_z(k) exp(+2 pi i k.m / M), m in I_N^2  Eq. NURSD1
 *
 * with theta_l = 2 pi (x_l - c) / (M delta), M = 2N, k in I_M^2 =
 * {-M/2..M/2-1}^2 and Ghat_{z,f} the M x M DFT of G = exp(+i k_f r)/r,
 * r = sqrt(|j delta|^2 + z^2) (Eq. RSD_conv).
 *
 * Conventions for every entry point:
 *  - All arrays are row-major with the LAST index contiguous; complex values
 *    are interleaved (re, im) float pairs (nursd_c64).
 *  - "d_" pointers are device pointers on the plan's device, "h_" pointers
 *    are host pointers.  The caller owns every input and output buffer; the
 *    plan owns its workspace and tables.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered and asynchronous: nothing synchronises the host except
 *    nursd_plan_create (which builds the transfer-function table) and
 *    nursd_sync_status.
 *  - Errors are returned as nursd_status values; no exception crosses the
 *    ABI.  Argument errors are detected on the host before any launch.
 *  - One plan must not be used from two host threads at once; distinct
 *    plans are independent.
 */
#ifndef NURSD_H
#define NURSD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nursd_plan_s* nursd_plan_t;
typedef struct {
  float re, im;
} nursd_c64;
/* A cudaStream_t passed as an opaque pointer. */
typedef void* nursd_stream_t;

typedef enum {
  NURSD_OK = 0,
  NURSD_ERR_INVALID_ARG = 1,        /* bad pointer, size or plan state      */
  NURSD_ERR_OOM = 2,                /* device allocation failed              */
  NURSD_ERR_CUDA = 3,               /* a CUDA call or launch failed          */
  NURSD_ERR_TIMEOUT = 4,            /* a bounded device wait gave up         */
  NURSD_ERR_UNSUPPORTED = 5,        /* size or feature not built             */
  NURSD_ERR_POINT_OUT_OF_RANGE = 6  /* a sample lies outside the aperture    */
} nursd_status;

/* Plan flags. */
#define NURSD_OUTPUT_MAGNITUDE 0x1u /* nursd_forward* write |V| (float32) instead of V */
#define NURSD_ENABLE_ADJOINT 0x2u   /* also build the transposed table used by nursd_adjoint and
                                       nursd_grad_points (doubles the table memory; Z <= 256) */
#define NURSD_CONFOCAL 0x4u         /* confocal acquisition (Supp., confocal systems): each relay
                                       point both illuminates and detects, the round trip doubles the
                                       phase, so every table uses the kernel e^{+i 2 k r} / r.
                                       nursd_forward_illuminated is unsupported on such plans. */

/*
 * Plan descriptor.  Geometry of Sec. 3.1 / Eq. 4: an N x N output lattice of
 * pitch `pitch` (metres) centred at (center_x, center_y) on the relay plane
 * z = 0, Z depth planes, F phasor frequencies.
 */
typedef struct {
  int32_t N;                 /* output lattice size, power of two, 8..512          */
  double pitch;              /* lattice pitch delta [m]                            */
  double center_x, center_y; /* lattice centre c [m]                               */
  int32_t Z;                 /* number of depth planes, 1..4096                    */
  const double* h_depths;    /* [Z] plane depths z_v > 0 [m] (copied)              */
  int32_t F;                 /* number of frequencies, 1..256                      */
  const double* h_omega;     /* [F] angular frequencies w_f [rad/s] (copied)       */
  const double* h_weight;    /* [F] filter weights w_f, or NULL: the Gaussian of    */
                             /* Eq. PFPacket from lambda_c (all ones if it is 0)  */
  int32_t T;                 /* histogram bins (0 = no histogram input)            */
  double t0, dt;             /* time of bin 0 and bin width [s]                    */
  int32_t upsample;          /* NUFFT oversampling sigma (only 2 is built)         */
  int32_t kernel_width;      /* ES kernel width w, 4..8 (6 gives ~1e-5)            */
  uint32_t flags;            /* NURSD_* flags                                      */
  int32_t max_points;        /* capacity for relay samples L                       */
  const double* h_srsd_pitch; /* [Z] SRSD output pitch delta_o(z) per depth [m] (copied),
                                 or NULL: no SRSD tables are built                  */
  int32_t max_batch;          /* capacity of nursd_forward_batched (0: not used), <= 256 */
  double lambda_c;            /* central wavelength [m] of the phasor-field band-pass: with
                                 h_weight NULL, w_f = exp(-(w_f - w_c)^2 / (2 (w_c / 5)^2)),
                                 w_c = 2 pi c / lambda_c (as nursd_phasor_frequencies); 0: none */
} nursd_desc;

/* One reconstruction of a batch: L relay samples d_xy [L][2], histograms
 * d_hist [L][T], output d_out [Z][N][N] (complex64 or magnitude float32). */
typedef struct {
  int32_t L;
  const float* d_xy;
  const float* d_hist;
  void* d_out;
} nursd_batch_item;

/* Text for a status code (static storage). */
const char* nursd_status_string(int status);

/*
 * Phasor-field frequencies and weights of Eq. PFPacket (host only): F
 * contiguous bins of a zero-padded length-t_pad DFT of step dt around
 * f_c = c / lambda_c, w_f = 2 pi (f0 + f) / (t_pad dt) with
 * f0 = round(f_c t_pad dt) - F/2, and Gaussian weights
 * exp(-(w - w_c)^2 / (2 sigma^2)), sigma = w_c / 5.  Writes F values to each
 * of h_omega and h_weight.  INVALID_ARG for non-positive inputs.
 */
int nursd_phasor_frequencies(double lambda_c, double dt, int32_t t_pad, int32_t F, double* h_omega,
                             double* h_weight);

/*
 * Create a plan: validates the descriptor, allocates the workspace on the
 * current device and builds, on `stream`, the transfer-function table
 * Ghat_{z,f} of Eq. 4 (FP64 phase k r reduced mod 2 pi, FP32 DFT), stored once
 * per class of the 8-fold symmetry Ghat(kx,ky) = Ghat(+-kx,+-ky) = Ghat(ky,kx).
 * Synchronises `stream` before returning.  On error *out is NULL and nothing
 * is leaked.
 */
int nursd_plan_create(const nursd_desc* desc, nursd_stream_t stream, nursd_plan_t* out);
/* The same call under the name of the interface statement (nursd_plan(desc, stream, &plan)). */
int nursd_plan(const nursd_desc* desc, nursd_stream_t stream, nursd_plan_t* out);

/* Free a plan and all its device memory (NULL is accepted). */
int nursd_plan_destroy(nursd_plan_t plan);

/* Device bytes held by the plan (tables + workspace), or -1 for NULL. */
int64_t nursd_plan_bytes(nursd_plan_t plan);

/* Sizes the plan derived: M = 2N, the fine-grid size, the number of
 * symmetry classes of the transfer-function table. Any pointer may be NULL. */
int nursd_plan_dims(nursd_plan_t plan, int32_t* M, int32_t* fine_n, int32_t* n_classes);

/*
 * Set the relay samples (Sec. 6: an unordered list rescaled to [-pi, pi)^2):
 * d_xy is [L][2] float32 metres on the relay plane, L <= max_points.  Computes
 * each sample's fine-grid footprint and ES weights and sorts the samples
 * (stably) into spreading tiles.  The plan copies what it needs; the caller
 * keeps d_xy.  A sample with |x - c| > N delta / 2 in either axis is an error:
 * its weights are zeroed and NURSD_ERR_POINT_OUT_OF_RANGE is reported by the
 * next nursd_sync_status.
 */
int nursd_set_points(nursd_plan_t plan, int32_t L, const float* d_xy, nursd_stream_t stream);

/*
 * Temporal transform (Eq. PF_Response with the filter of Eq. PFPacket):
 * d_hist [L][T] float32 histograms -> d_phasor [L][F] complex64,
 * P[l][f] = w_f sum_n h[l][n] exp(-i w_f (t0 + n dt)).  Needs T > 0 in the
 * descriptor; L <= max_points.  Independent of nursd_set_points.
 */
int nursd_temporal_dft(nursd_plan_t plan, int32_t L, const float* d_hist, nursd_c64* d_phasor,
                       nursd_stream_t stream);

/*
 * NUFFT type 1 of the current relay samples (Sec. 6: spread with the ES
 * kernel, FFT, deconvolve): d_phasor [L][F] -> d_spectrum [M][M][F] with
 * d_spectrum[ky+M/2][kx+M/2][f] ~= sum_l P[l][f] exp(-i (kx th_x + ky th_y)).
 * Requires nursd_set_points.
 */
int nursd_nufft1(nursd_plan_t plan, const nursd_c64* d_phasor, nursd_c64* d_spectrum,
                 nursd_stream_t stream);

/*
 * RSD propagation of a spectrum (Eq. NURSD1 after the NUFFT): frequency sum of
 * U_f Ghat_{z,f} and inverse DFT cropped to the N x N lattice:
 * d_spectrum [M][M][F] -> d_out [Z][N][N] (complex64, or float32 magnitude
 * with NURSD_OUTPUT_MAGNITUDE).
 */
int nursd_propagate(nursd_plan_t plan, const nursd_c64* d_spectrum, void* d_out, nursd_stream_t stream);

/*
 * Full NURSD-1 forward from phasors: nursd_nufft1 then nursd_propagate.
 * d_phasor [L][F] -> d_out [Z][N][N].  Requires nursd_set_points.
 */
int nursd_forward_phasor(nursd_plan_t plan, const nursd_c64* d_phasor, void* d_out,
                         nursd_stream_t stream);

/*
 * Full NURSD-1 forward from histograms (temporal transform, NUFFT-1, RSD,
 * frequency sum, inverse DFT): d_hist [L][T] float32 -> d_out [Z][N][N], L the
 * count given to nursd_set_points.
 */
int nursd_forward(nursd_plan_t plan, const float* d_hist, void* d_out, nursd_stream_t stream);

/*
 * The whole NURSD-1 reconstruction from raw inputs (Eq. NURSD1 with the frequency
 * integral of Eq. PF_RSD_Defn): nursd_set_points(L, d_xy) followed by
 * nursd_forward(d_hist, d_out), with the same result bit for bit.  The sample
 * sort (NUFFT-1 step 1, Sec. 6) runs on a plan-internal stream beside the
 * temporal transform and is joined before the spread; all work is ordered on
 * `stream` as usual: it starts after earlier work on `stream`, and later work on
 * `stream` starts after its last read of d_xy and d_hist.  The plan keeps the
 * points (later calls see L samples).  d_xy [L][2] float32 (8-byte aligned),
 * d_hist [L][T] float32 (16-byte aligned), d_out as for nursd_forward.
 * Returns NURSD_ERR_INVALID_ARG for bad arguments, NURSD_ERR_CUDA on a failed
 * stream, event or launch call.
 */
int nursd_reconstruct(nursd_plan_t plan, int32_t L, const float* d_xy, const float* d_hist, void* d_out,
                      nursd_stream_t stream);

/*
 * NURSD-2/3 output (Eqs. NURSD2 and NURSD3): the forward from phasors evaluated
 * at arbitrary voxels of each depth plane instead of the lattice:
 *   V_z(x_v) = M^-2 sum_k Y_z(k) exp(+i k . theta_v),  theta_v = 2 pi (x_v - c) / (M delta),
 * with Y_z as in nursd_propagate.  Computed by type-2 NUFFT (deconvolve,
 * inverse fine-grid FFT, ES interpolation).  d_vox_xy [Z][K][2] float32
 * metres (K voxels per plane, plane z at depth z_z), d_out [Z][K] complex64.
 * Voxels outside |x - c| <= N delta / 2 give 0 and set the out-of-range
 * status bit.  Requires nursd_set_points.
 */
int nursd_forward_points(nursd_plan_t plan, const nursd_c64* d_phasor, int32_t K, const float* d_vox_xy,
                         nursd_c64* d_out, nursd_stream_t stream);

/*
 * Adjoint of nursd_forward_phasor (type 2 is the adjoint of type 1, Sec. 6):
 *   P^H[l][f] = sum_k R_f(k) exp(+i k . theta_l),
 *   R_f(k) = sum_z conj(Ghat_{z,f}(k)) M^-2 sum_{m in I_N^2} V_z[m] exp(-2 pi i k.m / M).
 * d_vol [Z][N][N] complex64 -> d_phasor [L][F] complex64 at the current relay
 * samples.  Needs a plan created with NURSD_ENABLE_ADJOINT.
 */
int nursd_adjoint(nursd_plan_t plan, const nursd_c64* d_vol, nursd_c64* d_phasor, nursd_stream_t stream);

/*
 * Gradients of a real loss L(V), V = A(P, x) the complex NURSD-1 forward, given
 * d_w = 2 dL/d conj(V) [Z][N][N] (for L = ||V - V_t||^2, d_w = 2 (V - V_t)):
 *   d_grad_phasor [L][F] = A^H w                           (conjugate-Wirtinger
 *                                                            gradient w.r.t. P)
 *   d_grad_xy[l] = Re sum_f P[l][f] conj(d (A^H w)[l][f] / d(x_l, y_l))   [L][2]
 * The position derivative is the spectral one: d/dx of sum_k R_f(k) e^{ik.theta_l}
 * is i (2 pi / (M delta)) times the type-2 sum of kx R_f (likewise y), each
 * evaluated by the same NUFFT type 2 as the value, so it carries the value's
 * accuracy.  Either output may be NULL (not both); d_phasor is needed for
 * d_grad_xy.  Needs NURSD_ENABLE_ADJOINT.
 */
int nursd_grad_points(nursd_plan_t plan, const nursd_c64* d_w, const nursd_c64* d_phasor, nursd_c64* d_grad_phasor,
                      float* d_grad_xy, nursd_stream_t stream);

/*
 * Scaled RSD (Sec. 4, Eq. SRSD_conv with the SFFT of Supp. A.1, applied to a
 * non-uniform acquisition as in Supp. C): plane z is reconstructed on the
 * lattice c + delta_o(z) I_N^2 (delta_o from the descriptor's h_srsd_pitch,
 * scale s_z = delta_o(z) / delta, any positive value).  From the NUFFT-1
 * spectrum U_f the gridded input u_f = M^-2 IDFT_M[U_f] (on I_M^2, pitch delta)
 * is formed, then per depth and frequency the scaled DFT
 *   Phat_{z,f}(kappa) = sum_{n in I_M^2} u_f[n] exp(-2 pi i kappa.n / (M s_z)),
 * the frequency sum Y_z = sum_f Phat_{z,f} Ghat^(s_z)_{z,f} with G sampled at
 * pitch s_z delta, and the inverse DFT cropped to I_N^2:
 *   V_z[m] = M^-2 sum_kappa Y_z(kappa) exp(+2 pi i kappa.m / M).
 * Depths with s_z >= 1 take the scaled DFT as an ES interpolation of one
 * oversampled 2M x 2M spectrum of u_f / psi_hat shared by all depths (to the
 * NUFFT kernel's accuracy), all of them in one launch fused with the frequency
 * sum; depths with s_z < 1 take Bluestein's chirp-z (separable, convolution
 * length 2M).
 * d_phasor [L][F] -> d_out [Z][N][N] (complex64, or |V| with
 * NURSD_OUTPUT_MAGNITUDE).  Needs h_srsd_pitch at plan creation and
 * nursd_set_points.
 */
int srsd_forward(nursd_plan_t plan, const nursd_c64* d_phasor, void* d_out, nursd_stream_t stream);

/*
 * srsd_forward with the output pitch of each depth given at the call, as in the interface
 * statement (srsd_forward(plan, pitch_per_depth, in, out, stream)): h_pitch [Z] host, metres,
 * each > 0.  When the pitches differ from the plan's current SRSD pitches (or the plan was
 * created without h_srsd_pitch) the scaled table, the chirps and the interpolation taps are
 * rebuilt first: that call allocates on first use and synchronises like nursd_plan_create, so
 * only calls with unchanged pitches can be captured in a CUDA graph.  Then as srsd_forward.
 */
int srsd_forward_at(nursd_plan_t plan, const double* h_pitch, const nursd_c64* d_phasor, void* d_out,
                    nursd_stream_t stream);

/*
 * NU-SFFT (Supp. C, SRSD on non-uniform acquisition schemes: the fusion the
 * paper leaves to future work): the scaled DFT taken at the relay samples
 * themselves instead of a gridded input,
 *   Phat_{z,f}(kappa) = sum_l P[l][f] exp(-i kappa . theta_l / s_z),
 * then the frequency sum with Ghat^(s_z) and the inverse DFT crop as in
 * srsd_forward (the same output lattices).  Computed as the ES spread of the
 * samples, one FFT of the whole 2M x 2M grid divided by psi_hat in space, and per
 * depth ES taps at kappa / s_z divided by psi_hat(kappa / s_z), fused with the
 * contraction.  On the input lattice it equals srsd_forward; off it, it avoids
 * the band-limited gridding of u_f.  Every scale must be >= 1
 * (NURSD_ERR_UNSUPPORTED otherwise).  The first call allocates the NU-SFFT
 * tables and a [W][2M][F] buffer (W the spread window) and uploads the tables;
 * make it before any stream capture.  Needs h_srsd_pitch and nursd_set_points.
 */
int srsd_forward_nonuniform(nursd_plan_t plan, const nursd_c64* d_phasor, void* d_out, nursd_stream_t stream);

/*
 * SRSD + NURSD-2 (Eq. NURSD2_SRSD): the scaled spectra of srsd_forward
 *   Y^S_z(kappa) = sum_f Phat_{z,f}(kappa) Ghat^(s_z)_{z,f}(kappa)
 * evaluated at arbitrary voxels of each plane's scaled lattice by type 2:
 *   V_z(x_v) = M^-2 sum_kappa Y^S_z(kappa) exp(+i kappa . theta_v),
 *   theta_v = 2 pi (x_v - c) / (M s_z delta),
 * so voxels c + s_z delta m (m in I_N^2) give srsd_forward's output.
 * d_vox_xy [Z][K][2] float32 metres, d_out [Z][K] complex64.  Voxels outside
 * |x - c| <= N s_z delta / 2 give 0 and set the out-of-range status bit.
 * Needs h_srsd_pitch at plan creation and nursd_set_points.
 */
int srsd_forward_points(nursd_plan_t plan, const nursd_c64* d_phasor, int32_t K, const float* d_vox_xy,
                        nursd_c64* d_out, nursd_stream_t stream);

/*
 * Single-illumination reconstruction (Eq. PF_RSD_Defn for one illumination
 * point x_p): each frequency's reconstruction
 *   V_{z,f}[m] = M^-2 sum_k U_f(k) Ghat_{z,f}(k) exp(+2 pi i k.m / M),  m in I_N^2,
 * weighted by the illumination phase mask before the frequency sum:
 *   V_z[m] = sum_f exp(+i k_f |x_p - x_v|) V_{z,f}[m],
 *   x_v = (c_x + m_x delta, c_y + m_y delta, z_z),  k_f = w_f / c.
 * The mask cancels the delay of the path x_p -> x_v (the temporal transform's
 * e^{-i w t} convention), as the propagation kernel cancels the path back to
 * the relay.  h_illum: host [3] doubles (x, y, z) metres in the relay frame
 * (relay plane z = 0), read during the call.  d_phasor [L][F] -> d_out
 * [Z][N][N] complex64.  Requires nursd_set_points.  Depths are processed in
 * groups.  When Z % 4 == 0, F is even and M is 512 or 1024, a group is 4
 * depths (C = 4 F channels) whose products U_f Ghat_{z,f} are formed inside
 * the first inverse pass; otherwise a group is min(Z, max(1, 512 / F)) depths
 * and the products are written out first.  The first call of either
 * per-frequency form allocates the plan's workspace for them, about
 * 8 C (M N + N^2) bytes (plus 8 C M^2 without the in-pass products), and
 * uploads from host memory: neither call is capturable in a CUDA graph.
 */
int nursd_forward_illuminated(nursd_plan_t plan, const double* h_illum, const nursd_c64* d_phasor, nursd_c64* d_out,
                              nursd_stream_t stream);

/*
 * Time-resolved frames of the virtual wave (Eq. Video_Voxel_Freq_Offset): the
 * per-frequency reconstructions V_{z,f} (as in nursd_forward_illuminated)
 * summed with exp(+i w_f t) for each of n_frames times t (seconds on the
 * measurement's clock, the same origin as the descriptor's t0):
 *   frames[t][z][m] = sum_f exp(+i w_f t) V_{z,f}[m].
 * No illumination mask: a scatterer lights up when the virtual wave from the
 * illumination point reaches it.  h_times: host [n_frames], 1 <= n_frames <=
 * 4096.  d_phasor [L][F] -> d_out [n_frames][Z][N][N] complex64.  Requires
 * nursd_set_points; workspace and capture as for nursd_forward_illuminated.
 */
int nursd_transient_frames(nursd_plan_t plan, int32_t n_frames, const double* h_times, const nursd_c64* d_phasor,
                           nursd_c64* d_out, nursd_stream_t stream);

/*
 * B independent reconstructions with their own relay samples and histograms
 * (uneven L_b <= max_points), sharing the plan's geometry and transfer table:
 * for each item, what nursd_set_points + nursd_forward compute.  The temporal
 * transforms of all items are one persistent launch whose CTAs take 128-row
 * tiles of the ragged batch from a device work counter; the contraction is one
 * launch over all items that reads each table block from HBM once.  h_items is
 * a host array read during the call.  Allocates nothing, so the call can be
 * captured in a CUDA graph by the caller.  B <= max_batch.
 */
int nursd_forward_batched(nursd_plan_t plan, int32_t B, const nursd_batch_item* h_items, nursd_stream_t stream);

/*
 * Stage profiling.  Stages of the forward path, each one or more kernel
 * launches: relay-sample preparation and sort, temporal transform, spread,
 * FFT along x, FFT along y with deconvolution, transfer-function contraction,
 * inverse FFT along kx, inverse FFT along ky with crop.
 */
typedef enum {
  NURSD_STAGE_POINTS = 0,
  NURSD_STAGE_TEMPORAL = 1,
  NURSD_STAGE_SPREAD = 2,
  NURSD_STAGE_FFT_X = 3,
  NURSD_STAGE_FFT_Y = 4,
  NURSD_STAGE_CONTRACT = 5,
  NURSD_STAGE_IFFT_X = 6,
  NURSD_STAGE_IFFT_Y = 7,
  NURSD_STAGE_SRSD = 8, /* scaled transforms and per-depth contractions of srsd_forward */
  NURSD_STAGE_PER_FREQUENCY = 9, /* per-depth products and weighted frequency sums of the per-frequency forms */
  NURSD_NUM_STAGES = 10
} nursd_stage;

/*
 * enable != 0: from now on every stage brackets its launches with a pair of
 * CUDA events recorded on the caller's stream; enable == 0 stops recording.
 * Either way the recorded events are discarded.  While the stream is being
 * captured into a CUDA graph the pair is recorded as two event-record nodes
 * of the graph, so each replay of that graph times the stage again (one pair
 * per captured stage execution: capture a graph per replay whose times are
 * wanted, then read them after the replays).
 */
int nursd_profile_enable(nursd_plan_t plan, int enable);

/*
 * As nursd_profile_enable(plan, 1) for the stages whose bit (1u << stage) is
 * set in stage_mask only (0: recording off).  A single stage brackets fewer
 * launches than every stage would, so it perturbs the timed sequence less.
 */
int nursd_profile_select(nursd_plan_t plan, uint32_t stage_mask);

/*
 * For stage `stage`: *h_ms = summed device time of the launches recorded
 * since profiling was enabled (or last read), *h_count = number of recorded
 * stage executions.  Synchronises on the recorded events; resets them.
 */
int nursd_profile_read(nursd_plan_t plan, int stage, double* h_ms, int64_t* h_count);

/* Number of kernel launches the plan has issued since it was created. */
int64_t nursd_launch_count(nursd_plan_t plan);

/*
 * NUFFT type 1 that allocates nothing.  The paper has no counterpart: this is
 * a library facility.  Some callers cannot call cudaMalloc at all -- engines
 * that own every byte of device memory through a pre-reserved pool, and
 * plugins running inside them, where an extra allocation would synchronise the
 * device or escape the pool.  For them this computes what nursd_set_points
 * followed by nursd_nufft1 computes for a plan with the same N, pitch, centre,
 * kernel width and upsample 2: d_xy [L][2] float32 metres and d_phasor [L][F]
 * complex64 in, d_spectrum [M][M][F] complex64 out (M = 2N), all owned by the
 * caller.  No plan is needed and no device memory is allocated or freed.
 *
 * Its scratch is one fixed 24 MiB device array inside libnursd, present on
 * every GPU that loads the library until the process exits.  Per call it needs
 * 4M + 4 + L(24 + 16w) + 24 W tiles + 4 + 8 W F (W + M) bytes plus
 * alignment, with W = 16 ceil((2N + w + 2)/16) and tiles = W/16 (for example
 * N = 64, F = 32, L = 16,384 and w = 6 take about 12 MiB); larger requests
 * return NURSD_ERR_UNSUPPORTED before any device work.
 *
 * The first call on each device does a one-time set-up with that device
 * current: it looks up the array's device address and fills its fixed tables
 * with a small kernel, synchronising `stream`.  Make that first call before any
 * stream capture.  The set-up is repeated when the device's current context
 * is a new one (after cudaDeviceReset, say), whose copy of the array is new.  Every call shares the same array and leaves its contents
 * behind, so calls that overlap on the GPU (different streams, or different
 * host threads) race and must be serialised by the caller.  Samples outside
 * |x - c| <= N pitch / 2 get zero weight; they are not reported.
 */
int nursd_nufft1_noalloc(int32_t N, double pitch, double center_x, double center_y, int32_t kernel_width, int32_t L,
                         const float* d_xy, int32_t F, const nursd_c64* d_phasor, nursd_c64* d_spectrum,
                         nursd_stream_t stream);

/*
 * Synchronise `stream`, read and clear the plan's device error word.
 * Returns NURSD_OK, NURSD_ERR_POINT_OUT_OF_RANGE, NURSD_ERR_TIMEOUT (a bounded
 * device wait gave up) or NURSD_ERR_UNSUPPORTED (an SRSD tap table that the
 * interpolation kernels cannot follow; not produced by the plan's own tables), or, in
 * the checked build (libnursd_checked.so, compiled with -DNURSD_CHECKED), NURSD_ERR_CUDA
 * when a bounds check of a data-dependent index failed (the access was skipped).
 */
int nursd_sync_status(nursd_plan_t plan, nursd_stream_t stream);

/*
 * 3D NURSD for non-planar relay surfaces (Sec. 3D NURSD, Eq. 3D_NURSD with the 3D RSD of Eq. 3d_rsd;
 * stage 2 the standard RSD, Supp. C).  Relay samples lie at (x_l, y_l) with a height h_l = z_l - z0
 * above or below a reference plane z0; the plan's depths are then the distances of the voxel planes
 * from z0 (all > 0).  Stage 1 takes the field of every frequency on the N x N lattice of plane z0,
 *   W_f[m] = (M^2 Mz)^-1 sum_k U_f(k) Ghat3_f(k) exp(+2 pi i (kx mx + ky my) / M),  m in I_N^2,
 * with U_f the 3D type-1 sum of the samples at theta_l = (2 pi (x_l - c_x) / (M delta),
 * 2 pi (y_l - c_y) / (M delta), 2 pi h_l / (Mz dz)), k in I_M^2 x I_Mz, and Ghat3_f the 3D DFT of
 * G = exp(+i k_f r) / r on the offsets (j delta, jz dz), j in I_M^2, jz in I_Mz (G = 0 at the zero
 * offset); stage 2 propagates W_f from z0 to every plane and sums over frequency as nursd_forward_phasor
 * does for lattice samples.  Stage 1 is a 3D NUFFT: the ES spread along z (fine z grid of pitch dz / 2)
 * is applied per fine z cell to the phasors, each cell spread and transformed laterally like the planar
 * operator, then transformed along z.
 *
 * nursd_enable_3d: builds the 3D table (Mz a power of two, 8 <= Mz <= 512, Mz >= kernel_width + 2;
 *   allocates about M^2 F (2 Mz + kernel_width + 2) complex values); heights must satisfy
 *   |h| <= Mz dz / 4.  Synchronises the host like plan creation.  A second call with the same (dz, Mz)
 *   does nothing; other values give INVALID_ARG.
 * nursd_set_points_3d: d_xy [L][2] metres, d_h [L] heights (float32, device); sorts like
 *   nursd_set_points; a height beyond the range sets the out-of-range status bit and gets no weight.
 * nursd_forward_3d: d_phasor [L][F] -> d_out [Z][N][N] (complex64, or |V| with
 *   NURSD_OUTPUT_MAGNITUDE).  INVALID_ARG unless nursd_set_points_3d gave the current points.
 */
int nursd_enable_3d(nursd_plan_t plan, double dz, int32_t Mz, nursd_stream_t stream);
int nursd_set_points_3d(nursd_plan_t plan, int32_t L, const float* d_xy, const float* d_h, nursd_stream_t stream);
int nursd_forward_3d(nursd_plan_t plan, const nursd_c64* d_phasor, void* d_out, nursd_stream_t stream);

/*
 * Tunables of a plan (no counterpart in the paper: launch shapes of this library), set by the
 * autotuner of the Python package or by hand; they change only speed, never results beyond FP32
 * summation order.  NURSD_TUNE_SPREAD_ROWS: height in fine cells (4, 8 or 16) of the spread's tiles
 * (default 8).  NURSD_TUNE_BATCH_GROUPED: 1 (default) lets nursd_forward_batched run each stage as
 * one launch over a group of items when the items' outputs lie side by side (equally spaced, at least
 * one volume apart); 0 always takes the per-item form.  NURSD_TUNE_BATCH_STREAMS: streams (1 .. 16)
 * over which the per-item form runs its items' point sorts, spreads and FFT passes side by side
 * (default 4).  NURSD_TUNE_BATCH_GROUP: items per grouped launch, 1 .. the plan's capacity (default:
 * the capacity, max_batch or as many items as 8 GiB of item workspaces hold; 0 on plans without a
 * batch).  NURSD_TUNE_BATCH_TENSOR: 1 (default) runs the batched contraction (two or more items) as
 * tensor-core products per symmetry class where the shape allows (M a power of two, F a multiple of 8,
 * Z = 32, 64 or 128), 0 keeps the FP32 SIMT kernel; the two agree to FP32 rounding (the tensor form
 * splits each operand into tf32 head and tail and keeps the three leading products).
 * NURSD_TUNE_CONTRACT_TC: 0 (default) runs the contraction of a single reconstruction (and of the
 * adjoint) on the FP32 bulk-copy kernel; 1 runs it on the tensor cores where the shape allows (M a
 * power of two; forward: Z = 128, F a multiple of 16 up to 208, and a plan created with
 * NURSD_ENABLE_ADJOINT, whose [class][z][f] table copy the forward reads; adjoint: F = 128, Z a
 * multiple of 16 up to 208), else keeps the FP32 kernel.  With one reconstruction a class's product
 * has only 16 real output columns, and on this shape the tensor form is the slower of the two.  The
 * tensor form's error stays within about 3 (2K / 8) 2^-23 relative of the FP32 kernel's (K the
 * summed length: its accumulations are rounded toward zero).
 * nursd_plan_tune returns UNSUPPORTED for a value outside those sets, INVALID_ARG for an unknown
 * parameter.
 */
#define NURSD_TUNE_SPREAD_ROWS 0
#define NURSD_TUNE_BATCH_STREAMS 1
#define NURSD_TUNE_BATCH_GROUPED 2
#define NURSD_TUNE_BATCH_GROUP 3
#define NURSD_TUNE_BATCH_TENSOR 4
#define NURSD_TUNE_CONTRACT_TC 5
int nursd_plan_tune(nursd_plan_t plan, int32_t param, int32_t value);
int nursd_plan_get_tune(nursd_plan_t plan, int32_t param, int32_t* h_value);

/*
 * Test hooks (no counterpart in the paper), for the failure paths of this library.
 *
 * nursd_test_fail_allocation(after): process-wide; the after-th device allocation made by libnursd
 * from now on (1 = the next one) fails as if the device were out of memory, so that the call making
 * it returns NURSD_ERR_OOM and releases what it had allocated.  after <= 0 disarms the hook.
 *
 * nursd_test_set_wait_limit(polls, stream): on the current device, every plan's bulk-copy contraction
 * gives up its data waits after `polls` mbarrier polls (0: at the first wait, without polling; a
 * negative value restores the default of 2^22); a wait that runs out sets the plan's status word so
 * that nursd_sync_status returns NURSD_ERR_TIMEOUT, lets the warp's own copies in flight land (with
 * the default bound) and returns, leaving that call's output incomplete.  Stream-ordered on `stream`.
 */
int nursd_test_fail_allocation(int32_t after);
int nursd_test_set_wait_limit(int64_t polls, nursd_stream_t stream);

/*
 * Subsampled acquisition (Methods: Sampling Criteria for NLOS, Eq. upsample2): a relay grid may be
 * sampled D times more coarsely than the lattice when D < 2 |z_r - z_0| / |x_r - x_0| for the
 * scene's points; the compression keeps every D-th sample per axis and re-grids the kept phasors to
 * the full grid (nearest neighbour or linear) before a lattice reconstruction.  Plan-free and
 * allocation-free; stream-ordered.  Arrays are channel-last complex64: the grid
 * d_full [N][N][F] (row y, column x) and the kept samples d_kept [Nc][Nc][F], Nc = ceil(N / D), kept
 * sample (i, j) being grid sample (D i, D j).
 *
 * nursd_subsample: d_kept = d_full[::D, ::D].
 * nursd_upsample: d_full from d_kept; mode NURSD_UPSAMPLE_NEAREST: grid index n takes kept index
 *   min(ceil(n / D - 1/2), Nc - 1) per axis (halfway between two kept samples: the lower);
 *   NURSD_UPSAMPLE_LINEAR: separable linear interpolation between kept indices floor(n / D) and the
 *   next, holding the last kept value past it.
 * INVALID_ARG: N, F or D below 1, D > N, a null or misaligned (8-byte) pointer, an unknown mode.
 */
#define NURSD_UPSAMPLE_NEAREST 0
#define NURSD_UPSAMPLE_LINEAR 1
int nursd_subsample(int32_t N, int32_t F, int32_t D, const nursd_c64* d_full, nursd_c64* d_kept,
                    nursd_stream_t stream);
int nursd_upsample(int32_t N, int32_t F, int32_t D, int32_t mode, const nursd_c64* d_kept, nursd_c64* d_full,
                   nursd_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* NURSD_H */
