// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/litho.h"

namespace litho {

// thread-local error message behind litho_last_error()
void set_error(const char* fmt, ...);

#define LITHO_TRY_CUDA(expr)                                                                   \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      ::litho::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return LITHO_ECUDA;                                                                      \
    }                                                                                          \
  } while (0)

using cd = std::complex<double>;

// ---- per-stage device timing (prof.cpp) ------------------------------------------------------
enum Stage {
  kStageMaskSpectrum = 0,
  kStageStage1Fft,
  kStageStage2Fft,
  kStageGemmOperands,
  kStageStage2Gemm,
  kStageResist,
  kStageIltForward,
  kStageIltBackward,
  kStageIltReduce,
  kStageUpsample,
  kStageUpsampleResist,
  kStageContours,
  kStageEpe,
  kStageRaster,
  kStageCount
};
// Records a CUDA event pair around its lifetime on `st` when profiling is on.
class ProfScope {
 public:
  ProfScope(int stage, cudaStream_t st, int launches);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  int stage_;
  cudaStream_t st_;
  int launches_;
  void* a_ = nullptr;
};

// ---- host optics builder (optics.cpp) -------------------------------------------------------
struct SourcePoints {
  std::vector<double> sx, sy, w;  // units of NA/wavelength; sum w = 1
};
bool sample_source(const litho_optics& o, SourcePoints* out, std::string* why);
int band_crop(const litho_optics& o, const SourcePoints& s, int n, double pixel_nm);

struct FocusKernels {
  std::vector<double> lambda;  // [k], descending, 0 beyond rank
  std::vector<cd> phi;         // [k][C][C]
  int rank = 0;
  double trace = 0.0, gap = 0.0;
};
// Eigen-kernels of the TCC of one focus plane (Eqs. (2)-(3)).
bool build_focus_kernels(const litho_optics& o, const SourcePoints& s, int n, double pixel_nm, double z_nm, int k,
                         int crop, FocusKernels* out, std::string* why);
// Cyclic Jacobi for a Hermitian matrix (row-major, n x n, destroyed). Eigenvalues
// ascending in `ev` are not guaranteed: the caller sorts.  V columns = eigenvectors.
void hermitian_jacobi(std::vector<cd>& a, int n, std::vector<double>& ev, std::vector<cd>& v);

// ---- device data for the GEMM path --------------------------------------------------------
struct GemmOperands;  // gemm.cu

}  // namespace litho

struct litho_kernels {
  int n = 0, crop = 0, n_focus = 0, k = 0;
  double pixel_nm = 0.0;
  std::vector<int> rank;
  std::vector<double> lambda, trace, gap;  // [F*K], [F], [F]
  std::vector<double> phi_host;            // [F][K][C][C][2]
  float* d_lambda = nullptr;               // [F*K]
  float2* d_phi = nullptr;                 // [F][K][C][C]
  float2* d_tw = nullptr;                  // FFT twiddle table for N
  int nc = 0;                              // FP32 FFT coarse grid: smallest power of two >= 2 crop (0: not below N)
  float2* d_twc = nullptr;                 // FFT twiddle table for nc
  int nc_tc = 0;                           // tensor-core coarse grid: as nc, or 896 when 2 crop <= 896 < nc
  float2* d_twc_tc = nullptr;              // FFT twiddle table for nc_tc (d_twc when nc_tc == nc)
  float2* d_tw32 = nullptr;                // second-pass twiddles of the warp-per-row 1024-point stage 2
                                           // (when N or nc is 1024, else NULL)
  float2* d_phi_s = nullptr;               // sqrt(lam_fk) Phi_fk [F][K][C][C]: the aerial path's stage 1 on a
                                           // 1024-point grid, so that stage 2 sums |E|^2 unweighted (with d_tw32)
  float2* d_tw512 = nullptr;               // twiddles of the 512-point adjoint rows, two rows per warp
                                           // (when N or nc is 512, else NULL)
  litho::GemmOperands* gemm = nullptr;     // lazily built per precision
  int device = 0;
  // streams and events of the pipelined host-buffer path (created on first use)
  std::mutex host_mu;
  cudaStream_t host_streams[3] = {nullptr, nullptr, nullptr};  // input copies, kernels, output copies
  cudaEvent_t host_events[3] = {nullptr, nullptr, nullptr};
  // timing events of the host-buffer path (one start, three per chunk), grown on demand
  std::vector<cudaEvent_t> host_timing;
  std::vector<cudaEvent_t> host_sync;  // ordering events of the host-buffer path, three per chunk
};

namespace litho {

// Coarse grid for a band of C columns on an N grid (api.cpp): smallest power
// of two >= 2C, or with allow896 also 896; 0 when not below N.
int coarse_grid(int C, int N, bool allow896);

// Coarse evaluation grid of a precision's path (0 when it does not apply) and its twiddle table.
inline int coarse_n(const litho_kernels* h, litho_precision p) { return p == LITHO_PREC_FFT32 ? h->nc : h->nc_tc; }
inline const float2* coarse_tw(const litho_kernels* h, litho_precision p) {
  return p == LITHO_PREC_FFT32 ? h->d_twc : h->d_twc_tc;
}

// ---- launchers (fft.cu) ---------------------------------------------------------------------
// The N-entry per-pass twiddle table the FFT kernels expect (false if n unsupported).
bool fft_twiddle_table(int n, float2* out);
// Mask spectrum: m[b][n][n] -> mhat[b][C][C] = N^-2 DFT(m) on the crop.  rowbuf: [b][n][C].
// With `gain` [C] the stored value is mhat (1 + i gain[v] gain[u]) (blur channel, see fft.cu),
// or with gain_real mhat gain[v] gain[u] (the spectrum of the blurred plane).
cudaError_t launch_mask_spectrum(const float* m, int b, int n, int crop, const float2* tw, float2* rowbuf,
                                 float2* mhat, cudaStream_t st, const float* gain = nullptr, bool gain_real = false);
// Row pass of the mask spectrum alone: rowbuf[b][n][C] = row DFT of m, crop columns kept.
cudaError_t launch_mask_rows(const float* m, int b, int n, int crop, const float2* tw, float2* rowbuf, cudaStream_t st);
// Column pass of the interpolation from an nc grid to an n grid (interp.cu):
// q[p][n][c2] = inverse transform on n of the crop c2 of nc^-2 x forward
// transform on nc of rspec[p][nc][c2] (times 1 + i gain[v] gain[u] with gain).
bool interp_cols_supported(int nc, int n);
cudaError_t launch_interp_cols(const float2* rspec, int planes, int nc, int n, int c2, const float2* tw_nc,
                               const float2* tw_n, const float* gain, float2* q, cudaStream_t st);
// Stage 1 (band multiply + inverse DFT over v): for kernels phi[nk][C][C],
// t1[j][y][c] = sum_v mhat[v][c] phi_j[v][c] e^{+2 pi i v y/N}, j in [0, nk).
// phi == NULL transforms nk spectra mhat[j][C][C] themselves.  With kernels,
// `clips` spectra mhat[clips][C][C] are imaged in one launch; clip i writes
// t1[j + i nk].
cudaError_t launch_stage1_fft(const float2* mhat, const float2* phi, int nk, int n, int crop, const float2* tw,
                              float2* t1, cudaStream_t st, int clips = 1);
// Stage 2 FFT path: I[y][x] = dose * sum_j lam[j] |sum_c t1[j][y][c] e^{+2 pi i u_c x/N}|^2
// for each of `planes` planes; plane p takes lam[(p mod lam_period) nk ...]
// (lam_period <= 0: planes, no repetition).  With tw32 (the kernel set's
// d_tw32) a 1024-point row takes the warp-per-row radix-32 kernel, with
// tw512 (d_tw512) 512-point rows the two-rows-per-warp kernel.  folded (with
// tw32 only): the fields were made from sqrt(lam) Phi, so |E|^2 is summed
// without the weight (lam still marks the zero kernels, which are skipped).
// spec (with tw32 only): instead of the image, each image row's forward
// transform on the spec_crop frequencies |u| < spec_crop/2, laid out as
// launch_mask_rows writes them ([planes][n][spec_crop]); img is not written.
cudaError_t launch_stage2_fft(const float2* t1, const float* lam, int nk, int n, int crop, float dose,
                              const float2* tw, float* img, int planes, long long t1_plane_stride,
                              long long img_plane_stride, cudaStream_t st, int lam_period = 0,
                              const float2* tw32 = nullptr, const float2* tw512 = nullptr, bool folded = false,
                              float2* spec = nullptr, int spec_crop = 0);
// The warp-per-row stage 2 for 1024-point rows (stage2_w32.cu) and its
// second-pass twiddle table (31 x 32 entries w^(r l), r in [1, 32), l in [0, 32)).
bool stage2_w32_supported(int n, int crop);
// The two-rows-per-warp stage 2 for 512-point rows (twiddles: the kernel set's d_tw512).
bool stage2_w512_supported(int n, int crop);
cudaError_t launch_stage2_w512(const float2* t1, const float* lam, int nk, int n, int crop, float dose,
                               const float2* tw512, float* img, int planes, long long t1_plane, long long img_plane,
                               int lam_period, cudaStream_t st);
void stage2_w32_table(float2* out);
constexpr int kStage2W32TableLen = 31 * 32;
cudaError_t launch_stage2_w32(const float2* t1, const float* lam, int nk, int n, int crop, float dose,
                              const float2* tw2, float* img, int planes, long long t1_plane, long long img_plane,
                              int lam_period, cudaStream_t st, bool folded = false, float2* spec = nullptr,
                              int c2 = 0);

// A device-side delay of about `ms` milliseconds on `st` (util.cu): one
// thread spinning on the SM clock for a fixed number of cycles, which always
// ends.  The slow request of the serving tests.
cudaError_t launch_delay(cudaStream_t st, double ms);

// Twiddle table of the 512-point adjoint-rows kernel (ilt.cu): kAdj512TableLen entries.
constexpr int kAdj512TableLen = 31 * 16 + 15 * 32;
void adj512_table(float2* out);

// Device address of the per-clip FP64 losses inside an ILT workspace (ilt.cu).
double* ilt_loss_device(const litho_kernels* h, int b, void* workspace, size_t workspace_bytes);

// Channels 1 and 2 of Eq. (9) before normalisation (ilt.cu): for b targets
// at focus plane `focus`, x[c][1] = the aerial image and x[c][2] = the
// gradient of the plane's total intensity with respect to the mask pixels
// (x: [b][3][n][n]), in groups of clips; `coarse` evaluates the fields and
// the adjoint on the coarse grid.  Workspace: ai_channels_bytes(h, b).
size_t ai_channels_bytes(const litho_kernels* h, int b);
litho_status ai_channels(const litho_kernels* h, const float* target, int b, double dose, int focus, bool coarse,
                         float* x, void* workspace, cudaStream_t st);

// out[p][y][x] = scale Re(sum_c q[p][y][c] e^{+2 pi i u_c x/N}) for band rows q[p][N][C].
cudaError_t launch_band_rows_real(const float2* q, int planes, int n, int crop, float scale, const float2* tw,
                                  float* out, cudaStream_t st);

struct ResistTaps;
// gain[i] = sum_a g[a] cos(2 pi (i - crop/2) a / n): the blur's transfer function on the crop.
cudaError_t launch_blur_gain(const ResistTaps& taps, int n, int crop, float* gain, cudaStream_t st);
// Band rows carrying the blur channel: z = sum_c q[p][y][c] e^{+2 pi i u_c x/N};
// img = Re z (skipped when NULL), iblur = Im z, printed = [Im z >= threshold] (skipped when NULL).
// ILT forward end on the coarse grid, per pair of full-grid rows: blurred rows from the
// band rows, sigmoid resist, dL/dI and its row spectra on the crop (rowbuf, as
// launch_mask_rows), and one FP64 partial loss per row pair at partial[plane][pair]
// (planes x n/2 doubles).  Plane p uses target clip p / planes_per_clip.
cudaError_t launch_resist_grad_rows(const float2* band, int planes, int n, int crop, const float2* tw,
                                    const float* target, int planes_per_clip, float beta, float thr, float2* rowbuf,
                                    double* partial, cudaStream_t st);
// Column half of launch_mask_spectrum on row spectra already in rowbuf.
cudaError_t launch_mask_cols(const float2* rowbuf, int b, int n, int crop, const float2* tw, float2* mhat,
                             const float* gain, bool gain_real, cudaStream_t st);
cudaError_t launch_band_rows_resist(const float2* q, int planes, int n, int crop, const float2* tw, float threshold,
                                    float* img, float* iblur, uint8_t* printed, cudaStream_t st);

// ---- rectangle rasterisation (raster.cu) -----------------------------------------------------
long long raster_tiles_per_rect(int max_side);
size_t raster_workspace_bytes(int b, int n, long long max_rects, int max_side);
cudaError_t launch_raster(const float4* rects, const long long* rect_start, int b, long long max_rects,
                          int max_side, int n, float* mask, void* ws, cudaStream_t st);

// ---- contours and edge placement (contour.cu) -----------------------------------------------
size_t contour_workspace_bytes(int planes, int n);
cudaError_t launch_contours(const float* img, int planes, int n, float thr, float4* seg, int* cell_id,
                            long long capacity, long long* plane_start, void* ws, cudaStream_t st);
cudaError_t launch_epe(const float* img, int planes, int n, float pixel_nm, float thr, const float2* pts, int m,
                       float* epe, cudaStream_t st);
// Eq. (6) for all clips' points in one launch (points of clip c at [start[c], start[c+1])).
cudaError_t launch_epe_batch(const float* img, int clips, int planes, int n, float pixel_nm, float thr,
                             const float2* pts, const long long* start, long long m, float* epe, cudaStream_t st);
cudaError_t launch_epe_focus(const float* epe, int m, int f0, int fp, int fn, float tol_neg, float tol_pos,
                             float* avg, float* eff, cudaStream_t st);

// ---- resist (resist.cu) ---------------------------------------------------------------------
constexpr int kMaxResistRadius = 64;
struct ResistTaps {
  int radius;
  float g[2 * kMaxResistRadius + 1];
};
bool resist_taps(double sigma_nm, double pixel_nm, ResistTaps* t, std::string* why);
cudaError_t launch_resist(const float* img, int planes, int n, const ResistTaps& taps, float threshold, float* iblur,
                          uint8_t* printed, cudaStream_t st);

}  // namespace litho
