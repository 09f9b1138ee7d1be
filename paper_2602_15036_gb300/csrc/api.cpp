// C ABI entry points: kernel handles, aerial image, resist, error reporting.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "litho_internal.h"
#include "gemm.h"

namespace litho {

// Coarse evaluation grid for a field band of C columns on an N grid: the
// smallest power of two that is at least 2C, or with `allow896` also
// 896 = 16 x 8 x 7, or 0 when it is not below N.  The FP32 FFT path keeps
// powers of two: its 896-point transform issues more instructions per row
// than the 1024-point one (idle butterfly slots in the radix-16 and radix-8
// passes), so the smaller grid does not pay there; the tensor-core path's
// work scales with the grid's square.
int coarse_grid(int C, int N, bool allow896) {
  int nc = 32;
  while (nc < 2 * C) nc *= 2;
  if (allow896 && 2 * C <= 896 && 896 < nc) nc = 896;
  return nc < N ? nc : 0;
}

namespace {
thread_local char g_err[1024] = "";

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

bool valid_n(int n) {
  if (n < 32 || n > 2048) return false;
  return (n & (n - 1)) == 0;
}

// Bump allocator over the caller's workspace.
struct Carve {
  char* base;
  size_t cap, used = 0;
  Carve(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <class T>
  T* take(size_t count) {
    const size_t off = align_up(used);
    used = off + count * sizeof(T);
    return base ? reinterpret_cast<T*>(base + off) : nullptr;
  }
};

litho_status upload(litho_kernels* h) {
  const int F = h->n_focus, K = h->k, C = h->crop, N = h->n;
  LITHO_TRY_CUDA(cudaGetDevice(&h->device));
  std::vector<float> lam(size_t(F) * K);
  for (size_t i = 0; i < lam.size(); ++i) lam[i] = float(h->lambda[i]);
  std::vector<float2> phi(size_t(F) * K * C * C);
  for (size_t i = 0; i < phi.size(); ++i) phi[i] = make_float2(float(h->phi_host[2 * i]), float(h->phi_host[2 * i + 1]));
  std::vector<float2> tw(N);
  if (!fft_twiddle_table(N, tw.data())) {
    set_error("no FFT plan for n = %d", N);
    return LITHO_EINVAL;
  }
  LITHO_TRY_CUDA(cudaMalloc(&h->d_lambda, lam.size() * sizeof(float)));
  LITHO_TRY_CUDA(cudaMalloc(&h->d_phi, phi.size() * sizeof(float2)));
  LITHO_TRY_CUDA(cudaMalloc(&h->d_tw, tw.size() * sizeof(float2)));
  LITHO_TRY_CUDA(cudaMemcpy(h->d_lambda, lam.data(), lam.size() * sizeof(float), cudaMemcpyHostToDevice));
  LITHO_TRY_CUDA(cudaMemcpy(h->d_phi, phi.data(), phi.size() * sizeof(float2), cudaMemcpyHostToDevice));
  LITHO_TRY_CUDA(cudaMemcpy(h->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice));
  // coarse grid: I has no frequency at or beyond C along either axis, so
  // nc >= 2C samples determine it exactly
  h->nc = coarse_grid(C, N, false);
  h->nc_tc = coarse_grid(C, N, true);
  for (int pass = 0; pass < 2; ++pass) {
    const int nc = pass ? h->nc_tc : h->nc;
    float2** dst = pass ? &h->d_twc_tc : &h->d_twc;
    if (!nc) continue;
    if (pass && nc == h->nc) {
      h->d_twc_tc = h->d_twc;
      continue;
    }
    std::vector<float2> twc(nc);
    fft_twiddle_table(nc, twc.data());
    LITHO_TRY_CUDA(cudaMalloc(dst, twc.size() * sizeof(float2)));
    LITHO_TRY_CUDA(cudaMemcpy(*dst, twc.data(), twc.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }
  if (N == 512 || h->nc == 512) {
    std::vector<float2> t512(kAdj512TableLen);
    adj512_table(t512.data());
    LITHO_TRY_CUDA(cudaMalloc(&h->d_tw512, t512.size() * sizeof(float2)));
    LITHO_TRY_CUDA(cudaMemcpy(h->d_tw512, t512.data(), t512.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }
  if (N == 1024 || h->nc == 1024) {
    // sqrt(lam_fk) Phi_fk for the aerial path's stage 1 (FP64 product, then rounded)
    std::vector<float2> phs(phi.size());
    const size_t cc = size_t(C) * C;
    for (size_t fk = 0; fk < size_t(F) * K; ++fk) {
      const double r = std::sqrt(std::max(0.0, h->lambda[fk]));
      for (size_t i = 0; i < cc; ++i) {
        const size_t e = fk * cc + i;
        phs[e] = make_float2(float(r * h->phi_host[2 * e]), float(r * h->phi_host[2 * e + 1]));
      }
    }
    LITHO_TRY_CUDA(cudaMalloc(&h->d_phi_s, phs.size() * sizeof(float2)));
    LITHO_TRY_CUDA(cudaMemcpy(h->d_phi_s, phs.data(), phs.size() * sizeof(float2), cudaMemcpyHostToDevice));
    std::vector<float2> t32(kStage2W32TableLen);
    stage2_w32_table(t32.data());
    LITHO_TRY_CUDA(cudaMalloc(&h->d_tw32, t32.size() * sizeof(float2)));
    LITHO_TRY_CUDA(cudaMemcpy(h->d_tw32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }
  return LITHO_OK;
}

}  // namespace

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

}  // namespace litho

using namespace litho;

#define LITHO_REQUIRE(cond, msg)       \
  do {                                 \
    if (!(cond)) {                     \
      set_error("%s", msg);            \
      return LITHO_EINVAL;             \
    }                                  \
  } while (0)

extern "C" {

const char* litho_last_error(void) { return g_err; }
const char* litho_version(void) { return "litho-gb300 0.1 (sm_103a)"; }

void litho_free_kernels(litho_kernels* h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  cudaFree(h->d_lambda);
  cudaFree(h->d_phi);
  cudaFree(h->d_tw);
  if (h->d_twc_tc != h->d_twc) cudaFree(h->d_twc_tc);
  cudaFree(h->d_twc);
  cudaFree(h->d_tw32);
  cudaFree(h->d_phi_s);
  cudaFree(h->d_tw512);
  for (auto& s : h->host_streams)
    if (s) cudaStreamDestroy(s);
  for (auto& e : h->host_events)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->host_timing) cudaEventDestroy(e);
  for (auto& e : h->host_sync) cudaEventDestroy(e);
  gemm_free_operands(h);
  cudaSetDevice(cur);
  delete h;
}

litho_status litho_make_kernels(const litho_optics* optics, int n, double pixel_nm, const double* defocus_nm,
                                int n_focus, int k, litho_kernels** out) {
  LITHO_REQUIRE(optics && out && defocus_nm, "null argument");
  *out = nullptr;
  LITHO_REQUIRE(valid_n(n), "n must be a power of two in [32, 2048]");
  LITHO_REQUIRE(pixel_nm > 0 && std::isfinite(pixel_nm), "pixel_nm must be > 0");
  LITHO_REQUIRE(n_focus >= 1 && n_focus <= 64, "n_focus must be in [1, 64]");
  LITHO_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
  LITHO_REQUIRE(optics->wavelength_nm > 0 && optics->na > 0 && optics->n_medium >= optics->na,
                "need wavelength > 0 and 0 < NA <= n_medium");
  for (int f = 0; f < n_focus; ++f) LITHO_REQUIRE(std::isfinite(defocus_nm[f]), "defocus must be finite");
  SourcePoints src;
  std::string why;
  if (!sample_source(*optics, &src, &why)) {
    set_error("%s", why.c_str());
    return LITHO_EINVAL;
  }
  const int crop = band_crop(*optics, src, n, pixel_nm);
  auto* h = new (std::nothrow) litho_kernels();
  if (!h) {
    set_error("host allocation failed");
    return LITHO_ENOMEM;
  }
  h->n = n;
  h->crop = crop;
  h->n_focus = n_focus;
  h->k = k;
  h->pixel_nm = pixel_nm;
  const size_t cc = size_t(crop) * crop;
  try {
    h->lambda.assign(size_t(n_focus) * k, 0.0);
    h->phi_host.assign(size_t(n_focus) * k * cc * 2, 0.0);
    for (int f = 0; f < n_focus; ++f) {
      FocusKernels fk;
      if (!build_focus_kernels(*optics, src, n, pixel_nm, defocus_nm[f], k, crop, &fk, &why)) {
        set_error("%s", why.c_str());
        delete h;
        return LITHO_EINVAL;
      }
      h->rank.push_back(fk.rank);
      h->trace.push_back(fk.trace);
      h->gap.push_back(fk.gap);
      for (int i = 0; i < k; ++i) {
        h->lambda[size_t(f) * k + i] = fk.lambda[i];
        for (size_t b = 0; b < cc; ++b) {
          const cd v = fk.phi[size_t(i) * cc + b];
          h->phi_host[((size_t(f) * k + i) * cc + b) * 2] = v.real();
          h->phi_host[((size_t(f) * k + i) * cc + b) * 2 + 1] = v.imag();
        }
      }
    }
  } catch (const std::bad_alloc&) {
    delete h;
    set_error("host allocation failed while building kernels");
    return LITHO_ENOMEM;
  }
  litho_status st = upload(h);
  if (st != LITHO_OK) {
    litho_free_kernels(h);
    return st;
  }
  *out = h;
  return LITHO_OK;
}

litho_status litho_tcc_kernels_host(const litho_optics* optics, int n, double pixel_nm, double defocus_nm, int k,
                                    int* crop, double* lambda_host, double* phi_host, int* rank, double* trace,
                                    double* gap) {
  LITHO_REQUIRE(optics && crop, "null argument");
  LITHO_REQUIRE(valid_n(n), "n must be a power of two in [32, 2048]");
  LITHO_REQUIRE(pixel_nm > 0 && std::isfinite(pixel_nm) && std::isfinite(defocus_nm), "bad pixel or defocus");
  LITHO_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
  LITHO_REQUIRE(optics->wavelength_nm > 0 && optics->na > 0 && optics->n_medium >= optics->na,
                "need wavelength > 0 and 0 < NA <= n_medium");
  SourcePoints src;
  std::string why;
  if (!sample_source(*optics, &src, &why)) {
    set_error("%s", why.c_str());
    return LITHO_EINVAL;
  }
  *crop = band_crop(*optics, src, n, pixel_nm);
  if (!phi_host) return LITHO_OK;
  LITHO_REQUIRE(lambda_host, "lambda_host required with phi_host");
  FocusKernels fk;
  try {
    if (!build_focus_kernels(*optics, src, n, pixel_nm, defocus_nm, k, *crop, &fk, &why)) {
      set_error("%s", why.c_str());
      return LITHO_EINVAL;
    }
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed while building kernels");
    return LITHO_ENOMEM;
  }
  for (int i = 0; i < k; ++i) lambda_host[i] = fk.lambda[i];
  for (size_t i = 0; i < fk.phi.size(); ++i) {
    phi_host[2 * i] = fk.phi[i].real();
    phi_host[2 * i + 1] = fk.phi[i].imag();
  }
  if (rank) *rank = fk.rank;
  if (trace) *trace = fk.trace;
  if (gap) *gap = fk.gap;
  return LITHO_OK;
}

litho_status litho_upload_kernels(int n, double pixel_nm, int n_focus, int k, int crop, const double* lambda_host,
                                  const double* phi_host, litho_kernels** out) {
  LITHO_REQUIRE(out && lambda_host && phi_host, "null argument");
  *out = nullptr;
  LITHO_REQUIRE(valid_n(n), "n must be a power of two in [32, 2048]");
  LITHO_REQUIRE(crop >= 32 && crop <= n && crop % 32 == 0, "crop must be a multiple of 32 in [32, n]");
  LITHO_REQUIRE(n_focus >= 1 && n_focus <= 64 && k >= 1 && k <= 1024, "bad n_focus or k");
  LITHO_REQUIRE(pixel_nm > 0, "pixel_nm must be > 0");
  for (long long i = 0; i < (long long)n_focus * k; ++i)
    LITHO_REQUIRE(lambda_host[i] >= 0.0 && std::isfinite(lambda_host[i]), "lambda must be finite and >= 0");
  auto* h = new (std::nothrow) litho_kernels();
  if (!h) return LITHO_ENOMEM;
  h->n = n;
  h->crop = crop;
  h->n_focus = n_focus;
  h->k = k;
  h->pixel_nm = pixel_nm;
  const size_t cc = size_t(crop) * crop;
  h->lambda.assign(lambda_host, lambda_host + size_t(n_focus) * k);
  h->phi_host.assign(phi_host, phi_host + size_t(n_focus) * k * cc * 2);
  for (int f = 0; f < n_focus; ++f) {
    int r = 0;
    double tr = 0.0;
    for (int i = 0; i < k; ++i) {
      r += h->lambda[size_t(f) * k + i] > 0.0;
      tr += h->lambda[size_t(f) * k + i];
    }
    h->rank.push_back(r);
    h->trace.push_back(tr);
    h->gap.push_back(0.0);
  }
  litho_status st = upload(h);
  if (st != LITHO_OK) {
    litho_free_kernels(h);
    return st;
  }
  *out = h;
  return LITHO_OK;
}

litho_status litho_kernels_info(const litho_kernels* h, int* n, int* crop, int* n_focus, int* k, int* rank_host,
                                double* lambda_host, double* trace_host, double* gap_host) {
  LITHO_REQUIRE(h, "null handle");
  if (n) *n = h->n;
  if (crop) *crop = h->crop;
  if (n_focus) *n_focus = h->n_focus;
  if (k) *k = h->k;
  for (int f = 0; f < h->n_focus; ++f) {
    if (rank_host) rank_host[f] = h->rank[f];
    if (trace_host) trace_host[f] = h->trace[f];
    if (gap_host) gap_host[f] = h->gap[f];
  }
  if (lambda_host) std::memcpy(lambda_host, h->lambda.data(), h->lambda.size() * sizeof(double));
  return LITHO_OK;
}

litho_status litho_kernels_grid(const litho_kernels* h, int* nc_fft, int* nc_tensor) {
  LITHO_REQUIRE(h, "null handle");
  if (nc_fft) *nc_fft = h->nc;
  if (nc_tensor) *nc_tensor = h->nc_tc;
  return LITHO_OK;
}

litho_status litho_kernels_phi(const litho_kernels* h, double* phi_host) {
  LITHO_REQUIRE(h && phi_host, "null argument");
  std::memcpy(phi_host, h->phi_host.data(), h->phi_host.size() * sizeof(double));
  return LITHO_OK;
}

// ---- aerial ------------------------------------------------------------------------------------------

// Workspace regions of litho_aerial.  The FP32 FFT path images `group`
// clips per launch (their stage-1 fields side by side in t1); the GEMM path
// images groups of gemm_group_clips().  With the coarse grid the fields are
// evaluated on nc x nc and `ic` holds a group's images until the
// interpolation (mask-spectrum kernels on a 2C crop, stage 1 over y, band
// rows over x) writes the N x N result; `gain` holds the blur's transfer
// function when the resist is fused into that interpolation.
struct AerialLayout {
  float2 *rowbuf = nullptr, *mhat = nullptr, *t1 = nullptr;
  void* gws = nullptr;
  float* ic = nullptr;
  float2 *rowbuf2 = nullptr, *spec = nullptr, *q = nullptr;
  float* gain = nullptr;
  int group = 1;
  size_t bytes = 0;
};

// Clips per FP32 stage launch: enough CTAs that the last wave is a small
// share of the launch, with the group's stage-1 fields within 2 GiB, and
// groups of equal size.
static int fft_group_clips(const litho_kernels* h, int b, bool coarse) {
  const size_t NE = coarse ? coarse_n(h, LITHO_PREC_FFT32) : h->n;
  const size_t per_clip = size_t(h->n_focus) * h->k * NE * h->crop * sizeof(float2);
  const size_t cap = std::max<size_t>(1, std::min<size_t>(64, (size_t(2) << 30) / per_clip));
  const size_t groups = (size_t(b) + cap - 1) / cap;
  return int((size_t(b) + groups - 1) / groups);
}

static AerialLayout aerial_layout(const litho_kernels* h, int b, litho_precision prec, bool coarse, void* ws) {
  Carve c(ws, 0);
  const size_t N = h->n, C = h->crop, F = h->n_focus, K = h->k, NE = coarse ? coarse_n(h, prec) : h->n;
  AerialLayout L;
  L.rowbuf = c.take<float2>(size_t(b) * N * C);
  L.mhat = c.take<float2>(size_t(b) * C * C);
  if (prec == LITHO_PREC_FFT32) {
    L.group = fft_group_clips(h, b, coarse);
    L.t1 = c.take<float2>(size_t(L.group) * F * K * NE * C);
  } else {
    L.gws = c.take<char>(gemm_workspace_bytes(h, prec, b, coarse));
    L.group = std::min(b, gemm_group_clips());
  }
  const size_t planes = size_t(L.group) * F;
  if (coarse) {
    L.ic = c.take<float>(planes * NE * NE);
    L.rowbuf2 = c.take<float2>(planes * NE * 2 * C);
    L.spec = c.take<float2>(planes * 4 * C * C);
    L.q = c.take<float2>(planes * N * 2 * C);
    L.gain = c.take<float>(2 * C);
  }
  L.bytes = align_up(c.used);
  return L;
}

static bool decode_precision(int raw, litho_precision* p, bool* coarse) {
  if ((raw & ~(0xFF | LITHO_GRID_COARSE)) != 0) return false;
  const int base = raw & 0xFF;
  if (base < LITHO_PREC_FFT32 || base > LITHO_PREC_FP16) return false;
  *p = static_cast<litho_precision>(base);
  *coarse = (raw & LITHO_GRID_COARSE) != 0;
  return true;
}

// Resist fused into the coarse-grid interpolation: outputs of plane p of the
// call at iblur + p N^2 and printed + p N^2 (printed may be NULL).
struct FusedResist {
  float threshold;
  float* iblur;
  uint8_t* printed;
};

// `planes` coarse images in L.ic -> N x N planes at `out` (plane offset `p0`
// of the call for the fused resist outputs).
// rows_done: stage 2 has already written the coarse images' row spectra to L.rowbuf2.
static litho_status upsample(const litho_kernels* h, litho_precision p, const AerialLayout& L, int planes, float* out,
                             const FusedResist* fr, size_t p0, cudaStream_t st, bool rows_done = false) {
  const int N = h->n, NC = coarse_n(h, p), C2 = 2 * h->crop;
  const float2* twc = coarse_tw(h, p);
  const float* gain = fr ? L.gain : nullptr;
  ProfScope ps(fr ? kStageUpsampleResist : kStageUpsample, st, rows_done ? 2 : 3);
  if (interp_cols_supported(NC, N)) {
    if (!rows_done) LITHO_TRY_CUDA(launch_mask_rows(L.ic, planes, NC, C2, twc, L.rowbuf2, st));
    LITHO_TRY_CUDA(launch_interp_cols(L.rowbuf2, planes, NC, N, C2, twc, h->d_tw, gain, L.q, st));
  } else {
    LITHO_TRY_CUDA(launch_mask_spectrum(L.ic, planes, NC, C2, twc, L.rowbuf2, L.spec, st, gain));
    LITHO_TRY_CUDA(launch_stage1_fft(L.spec, nullptr, planes, N, C2, h->d_tw, L.q, st));
  }
  if (!fr) {
    LITHO_TRY_CUDA(launch_band_rows_real(L.q, planes, N, C2, 1.0f, h->d_tw, out, st));
    return LITHO_OK;
  }
  const size_t nn = size_t(N) * N;
  LITHO_TRY_CUDA(launch_band_rows_resist(L.q, planes, N, C2, h->d_tw, fr->threshold, out, fr->iblur + p0 * nn,
                                         fr->printed ? fr->printed + p0 * nn : nullptr, st));
  return LITHO_OK;
}

litho_status litho_aerial_workspace_size(const litho_kernels* h, int b, litho_precision prec, size_t* bytes) {
  LITHO_REQUIRE(h && bytes, "null argument");
  LITHO_REQUIRE(b >= 1, "b must be >= 1");
  litho_precision p;
  bool coarse;
  LITHO_REQUIRE(decode_precision(int(prec), &p, &coarse), "unknown precision");
  *bytes = aerial_layout(h, b, p, coarse && coarse_n(h, p) > 0, nullptr).bytes;
  return LITHO_OK;
}

// Argument checks shared by litho_aerial and litho_aerial_resist; fills the
// decoded precision and the layout.
static litho_status aerial_prepare(const litho_kernels* h, const float* mask_dev, int b, double dose, int prec,
                                   float* intensity_dev, void* workspace_dev, size_t workspace_bytes,
                                   litho_precision* p, bool* coarse, AerialLayout* L) {
  LITHO_REQUIRE(h && mask_dev && intensity_dev && workspace_dev, "null argument");
  LITHO_REQUIRE(b >= 1, "b must be >= 1");
  LITHO_REQUIRE(std::isfinite(dose), "dose must be finite");
  LITHO_REQUIRE(decode_precision(prec, p, coarse), "unknown precision");
  *coarse = *coarse && coarse_n(h, *p) > 0;
  LITHO_REQUIRE((reinterpret_cast<uintptr_t>(workspace_dev) & 255) == 0, "workspace must be 256-byte aligned");
  LITHO_REQUIRE((reinterpret_cast<uintptr_t>(mask_dev) & 15) == 0 && (reinterpret_cast<uintptr_t>(intensity_dev) & 15) == 0,
                "mask and intensity must be 16-byte aligned");
  const size_t need = aerial_layout(h, b, *p, *coarse, nullptr).bytes;
  if (workspace_bytes < need) {
    set_error("workspace too small: %zu bytes given, %zu needed", workspace_bytes, need);
    return LITHO_ENOMEM;
  }
  if (*p != LITHO_PREC_FFT32) {
    litho_status s = gemm_supported(h, *p, *coarse);
    if (s != LITHO_OK) return s;
  }
  *L = aerial_layout(h, b, *p, *coarse, workspace_dev);
  return LITHO_OK;
}

// The aerial image of b clips; with `fr` (coarse grid only) the resist is
// computed inside the interpolation.
static litho_status aerial_run(const litho_kernels* h, const float* mask_dev, int b, double dose, litho_precision p,
                               bool coarse, float* intensity_dev, const AerialLayout& L, const FusedResist* fr,
                               cudaStream_t st) {
  const int N = h->n, C = h->crop, F = h->n_focus, K = h->k;
  {
    ProfScope ps(kStageMaskSpectrum, st, 2);
    LITHO_TRY_CUDA(launch_mask_spectrum(mask_dev, b, N, C, h->d_tw, L.rowbuf, L.mhat, st));
  }
  const int G = L.group;
  if (p != LITHO_PREC_FFT32) {
    for (int c0 = 0; c0 < b; c0 += G) {
      const int g = std::min(G, b - c0);
      float* dst = intensity_dev + size_t(c0) * F * N * N;
      litho_status s =
          gemm_aerial_group(h, L.mhat + size_t(c0) * C * C, g, float(dose), p, coarse, coarse ? L.ic : dst, L.gws, st);
      if (s != LITHO_OK) return s;
      if (coarse && (s = upsample(h, p, L, g * F, dst, fr, size_t(c0) * F, st)) != LITHO_OK) return s;
    }
    return LITHO_OK;
  }
  const int NE = coarse ? coarse_n(h, p) : N;
  const float2* tw = coarse ? coarse_tw(h, p) : h->d_tw;
  // On a 1024-point grid stage 1 takes sqrt(lam) Phi and the warp-per-row stage 2 sums |E|^2 unweighted
  const bool folded = h->d_phi_s && h->d_tw32 && stage2_w32_supported(NE, C);
  // with the warp-per-row stage 2 on the coarse grid, stage 2 writes the row spectra that the
  // interpolation's column pass reads, in place of the coarse images
  const bool rows_in_stage2 = coarse && folded && interp_cols_supported(NE, N);
  for (int c0 = 0; c0 < b; c0 += G) {
    const int g = std::min(G, b - c0);
    float* img = intensity_dev + size_t(c0) * F * N * N;
    {
      ProfScope ps(kStageStage1Fft, st, 1);
      LITHO_TRY_CUDA(launch_stage1_fft(L.mhat + size_t(c0) * C * C, folded ? h->d_phi_s : h->d_phi, F * K, NE, C, tw,
                                       L.t1, st, g));
    }
    {
      ProfScope ps(kStageStage2Fft, st, 1);
      LITHO_TRY_CUDA(launch_stage2_fft(L.t1, h->d_lambda, K, NE, C, float(dose), tw, coarse ? L.ic : img, g * F,
                                       (long long)K * NE * C, (long long)NE * NE, st, F, h->d_tw32, h->d_tw512,
                                       folded, rows_in_stage2 ? L.rowbuf2 : nullptr, 2 * C));
    }
    if (coarse) {
      litho_status s = upsample(h, p, L, g * F, img, fr, size_t(c0) * F, st, rows_in_stage2);
      if (s != LITHO_OK) return s;
    }
  }
  return LITHO_OK;
}

litho_status litho_aerial(const litho_kernels* h, const float* mask_dev, int b, double dose, litho_precision prec,
                          float* intensity_dev, void* workspace_dev, size_t workspace_bytes, void* stream) {
  litho_precision p;
  bool coarse;
  AerialLayout L;
  litho_status s =
      aerial_prepare(h, mask_dev, b, dose, int(prec), intensity_dev, workspace_dev, workspace_bytes, &p, &coarse, &L);
  if (s != LITHO_OK) return s;
  return aerial_run(h, mask_dev, b, dose, p, coarse, intensity_dev, L, nullptr, static_cast<cudaStream_t>(stream));
}

litho_status litho_aerial_resist(const litho_kernels* h, const float* mask_dev, int b, double dose,
                                 litho_precision prec, float* intensity_dev, double sigma_nm, double threshold,
                                 float* iblur_dev, uint8_t* printed_dev, void* workspace_dev, size_t workspace_bytes,
                                 void* stream) {
  LITHO_REQUIRE(iblur_dev, "null argument");
  LITHO_REQUIRE(std::isfinite(threshold), "threshold must be finite");
  litho_precision p;
  bool coarse;
  AerialLayout L;
  litho_status s =
      aerial_prepare(h, mask_dev, b, dose, int(prec), intensity_dev, workspace_dev, workspace_bytes, &p, &coarse, &L);
  if (s != LITHO_OK) return s;
  ResistTaps taps;
  std::string why;
  if (!resist_taps(sigma_nm, h->pixel_nm, &taps, &why)) {
    set_error("%s", why.c_str());
    return LITHO_EINVAL;
  }
  LITHO_REQUIRE(2 * taps.radius < h->n, "blur radius must be below n/2");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!coarse) {
    s = aerial_run(h, mask_dev, b, dose, p, coarse, intensity_dev, L, nullptr, st);
    if (s != LITHO_OK) return s;
    ProfScope ps(kStageResist, st, 1);
    LITHO_TRY_CUDA(launch_resist(intensity_dev, b * h->n_focus, h->n, taps, float(threshold), iblur_dev, printed_dev,
                                 st));
    return LITHO_OK;
  }
  {
    ProfScope ps(kStageUpsampleResist, st, 1);
    LITHO_TRY_CUDA(launch_blur_gain(taps, h->n, 2 * h->crop, L.gain, st));
  }
  const FusedResist fr{float(threshold), iblur_dev, printed_dev};
  return aerial_run(h, mask_dev, b, dose, p, coarse, intensity_dev, L, &fr, st);
}

// The host-buffer path images the batch in chunks of clips on three library
// streams: input copies, kernels (one chunk after another, as the device
// path runs them) and output copies, ordered by events, so that the copies
// of neighbouring chunks overlap the kernels.  Chunks alternate between two
// regions of the workspace.
static int host_chunk_clips(int b) { return b >= 4 ? std::min(8, (b + 3) / 4) : b; }

// Host timestamps of the last litho_aerial_host call (litho_host_trace_read):
// when each chunk's copies and launches were issued and how long the final
// wait took, to tell a host-side stall from a device-side one.
namespace {
struct HostTrace {
  std::mutex mu;
  std::vector<int> tags;
  std::vector<double> ms;
};
HostTrace g_host_trace;
double host_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

static size_t host_region_bytes(const litho_kernels* h, int cb, litho_precision prec) {
  size_t w = 0;
  if (litho_aerial_workspace_size(h, cb, prec, &w) != LITHO_OK) return 0;
  const size_t nn = size_t(h->n) * h->n, planes = size_t(cb) * h->n_focus;
  return align_up(w) + align_up(size_t(cb) * nn * sizeof(float)) + 2 * align_up(planes * nn * sizeof(float)) +
         align_up(planes * nn);
}

litho_status litho_aerial_host_workspace_size(const litho_kernels* h, int b, litho_precision prec, size_t* bytes) {
  LITHO_REQUIRE(h && bytes && b >= 1, "bad argument");
  size_t w = 0;
  litho_status s = litho_aerial_workspace_size(h, b, prec, &w);  // validates prec
  if (s != LITHO_OK) return s;
  const int cb = host_chunk_clips(b);
  *bytes = (cb < b ? 2 : 1) * host_region_bytes(h, cb, prec);
  return LITHO_OK;
}

litho_status litho_aerial_host(const litho_kernels* h, const float* mask_host, int b, double dose,
                               litho_precision prec, float* intensity_host, double sigma_nm, double threshold,
                               uint8_t* printed_host, void* workspace_dev, size_t workspace_bytes, void* stream) {
  LITHO_REQUIRE(h && mask_host && workspace_dev, "null argument");
  LITHO_REQUIRE(intensity_host || printed_host, "nothing to return: intensity_host and printed_host are both NULL");
  size_t need = 0;
  litho_status s = litho_aerial_host_workspace_size(h, b, prec, &need);
  if (s != LITHO_OK) return s;
  if (workspace_bytes < need) {
    set_error("workspace too small: %zu bytes given, %zu needed", workspace_bytes, need);
    return LITHO_ENOMEM;
  }
  const int cb = host_chunk_clips(b), F = h->n_focus;
  // Chunk starts: the first and the last chunk take 2 clips when the batch is long, so that
  // the one input copy and the one output copy that nothing overlaps are short; the others
  // take at most cb clips, as evenly as possible.
  std::vector<int> starts{0};
  {
    const bool ends = b >= 4 * cb;
    const int head = ends ? 2 : 0, tail = ends ? 2 : 0, mid = b - head - tail;
    if (head) starts.push_back(head);
    const int nmid = (mid + cb - 1) / cb;
    for (int i = 1; i <= nmid; ++i) starts.push_back(head + int((long long)mid * i / nmid));
    if (tail) starts.push_back(b);
  }
  const int chunks = int(starts.size()) - 1;
  const size_t region = host_region_bytes(h, cb, prec);
  std::vector<int> ttag;
  std::vector<double> tms;
  const double t_start = host_ms();
  auto mark = [&](int tag) {
    ttag.push_back(tag);
    tms.push_back(host_ms() - t_start);
  };
  size_t w = 0;
  litho_aerial_workspace_size(h, cb, prec, &w);
  w = align_up(w);
  const size_t nn = size_t(h->n) * h->n;
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  litho_kernels* hm = const_cast<litho_kernels*>(h);
  // concurrent host-path calls on one kernel set share its streams and events: one at a time
  std::lock_guard<std::mutex> lk(hm->host_mu);
  for (auto& st : hm->host_streams)
    if (!st) LITHO_TRY_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  if (!hm->host_events[0]) LITHO_TRY_CUDA(cudaEventCreateWithFlags(&hm->host_events[0], cudaEventDisableTiming));
  // per chunk: input copied, kernels done, outputs copied (ordering), and the same three for timing
  while (hm->host_sync.size() < size_t(3 * chunks)) {
    cudaEvent_t e;
    LITHO_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    hm->host_sync.push_back(e);
  }
  while (hm->host_timing.size() < size_t(1 + 3 * chunks)) {
    cudaEvent_t e;
    LITHO_TRY_CUDA(cudaEventCreate(&e));
    hm->host_timing.push_back(e);
  }
  cudaStream_t s_in = hm->host_streams[0], s_comp = hm->host_streams[1], s_out = hm->host_streams[2];
  auto ev_in = [&](int ci) { return hm->host_sync[3 * ci]; };
  auto ev_comp = [&](int ci) { return hm->host_sync[3 * ci + 1]; };
  auto ev_out = [&](int ci) { return hm->host_sync[3 * ci + 2]; };
  LITHO_TRY_CUDA(cudaEventRecord(hm->host_events[0], caller));
  for (cudaStream_t st : {s_in, s_comp, s_out}) LITHO_TRY_CUDA(cudaStreamWaitEvent(st, hm->host_events[0], 0));
  LITHO_TRY_CUDA(cudaEventRecord(hm->host_timing[0], s_in));
  for (int ci = 0; ci < chunks; ++ci) {
    const int c0 = starts[ci], nb = starts[ci + 1] - c0;
    const size_t planes = size_t(nb) * F;
    // chunks alternate between two workspace regions
    char* base = static_cast<char*>(workspace_dev) + (ci & 1) * (cb < b ? region : 0);
    float* dmask = reinterpret_cast<float*>(base + w);
    float* dimg = reinterpret_cast<float*>(base + w + align_up(size_t(cb) * nn * sizeof(float)));
    float* dblur =
        reinterpret_cast<float*>(reinterpret_cast<char*>(dimg) + align_up(size_t(cb) * F * nn * sizeof(float)));
    uint8_t* dpr =
        reinterpret_cast<uint8_t*>(reinterpret_cast<char*>(dblur) + align_up(size_t(cb) * F * nn * sizeof(float)));
    // input copy: the region's mask buffer is free once the kernels of chunk ci - 2 are done
    if (ci >= 2) LITHO_TRY_CUDA(cudaStreamWaitEvent(s_in, ev_comp(ci - 2), 0));
    LITHO_TRY_CUDA(cudaMemcpyAsync(dmask, mask_host + size_t(c0) * nn, size_t(nb) * nn * sizeof(float),
                                   cudaMemcpyHostToDevice, s_in));
    LITHO_TRY_CUDA(cudaEventRecord(ev_in(ci), s_in));
    LITHO_TRY_CUDA(cudaEventRecord(hm->host_timing[1 + 3 * ci], s_in));
    mark(ci * 8 + 0);
    // kernels, one chunk after another on one stream: after the input copy, and once the
    // region's output buffers have been copied out for chunk ci - 2
    LITHO_TRY_CUDA(cudaStreamWaitEvent(s_comp, ev_in(ci), 0));
    if (ci >= 2) LITHO_TRY_CUDA(cudaStreamWaitEvent(s_comp, ev_out(ci - 2), 0));
    if (printed_host)
      s = litho_aerial_resist(h, dmask, nb, dose, prec, dimg, sigma_nm, threshold, dblur, dpr, base, w, s_comp);
    else
      s = litho_aerial(h, dmask, nb, dose, prec, dimg, base, w, s_comp);
    if (s != LITHO_OK) return s;
    LITHO_TRY_CUDA(cudaEventRecord(ev_comp(ci), s_comp));
    LITHO_TRY_CUDA(cudaEventRecord(hm->host_timing[2 + 3 * ci], s_comp));
    mark(ci * 8 + 1);
    // output copies
    LITHO_TRY_CUDA(cudaStreamWaitEvent(s_out, ev_comp(ci), 0));
    if (printed_host)
      LITHO_TRY_CUDA(
          cudaMemcpyAsync(printed_host + size_t(c0) * F * nn, dpr, planes * nn, cudaMemcpyDeviceToHost, s_out));
    if (intensity_host)
      LITHO_TRY_CUDA(cudaMemcpyAsync(intensity_host + size_t(c0) * F * nn, dimg, planes * nn * sizeof(float),
                                     cudaMemcpyDeviceToHost, s_out));
    LITHO_TRY_CUDA(cudaEventRecord(ev_out(ci), s_out));
    LITHO_TRY_CUDA(cudaEventRecord(hm->host_timing[3 + 3 * ci], s_out));
    mark(ci * 8 + 2);
  }
  // the last output copy follows every earlier step on all three streams
  LITHO_TRY_CUDA(cudaStreamWaitEvent(caller, ev_out(chunks - 1), 0));
  mark(-1);  // all work issued; the wait starts
  LITHO_TRY_CUDA(cudaStreamSynchronize(caller));
  mark(-2);  // the wait ended
  for (int ci = 0; ci < chunks; ++ci)
    for (int k = 0; k < 3; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, hm->host_timing[0], hm->host_timing[1 + 3 * ci + k]) == cudaSuccess) {
        ttag.push_back(100 + ci * 8 + k);
        tms.push_back(ms);
      }
    }
  {
    std::lock_guard<std::mutex> tl(g_host_trace.mu);
    g_host_trace.tags.swap(ttag);
    g_host_trace.ms.swap(tms);
  }
  return LITHO_OK;
}

litho_status litho_host_trace_read(int max_events, int* tags, double* ms, int* count) {
  LITHO_REQUIRE(count && (max_events <= 0 || (tags && ms)), "null argument");
  std::lock_guard<std::mutex> tl(g_host_trace.mu);
  const int n = std::min<int>(std::max(0, max_events), int(g_host_trace.tags.size()));
  for (int i = 0; i < n; ++i) {
    tags[i] = g_host_trace.tags[i];
    ms[i] = g_host_trace.ms[i];
  }
  *count = int(g_host_trace.tags.size());
  return LITHO_OK;
}

litho_status litho_check_device(const litho_kernels* h, void* stream) {
  LITHO_REQUIRE(h, "null handle");
  return gemm_check_device(h, static_cast<cudaStream_t>(stream));
}

litho_status litho_selftest_wait_limit(const litho_kernels* h, double limit_ms, void* stream) {
  LITHO_REQUIRE(h, "null handle");
  LITHO_REQUIRE(limit_ms > 0 && limit_ms <= 2000, "limit_ms must be in (0, 2000]");
  return gemm_wait_selftest(h, limit_ms, static_cast<cudaStream_t>(stream));
}

// ---- resist ------------------------------------------------------------------------------------------

litho_status litho_resist(const float* intensity_dev, int planes, int n, double pixel_nm, double sigma_nm,
                          double threshold, float* iblur_dev, uint8_t* printed_dev, void* stream) {
  LITHO_REQUIRE(intensity_dev && iblur_dev, "null argument");
  LITHO_REQUIRE(planes >= 1 && n >= 32 && n % 32 == 0, "planes >= 1 and n a multiple of 32 required");
  LITHO_REQUIRE(std::isfinite(threshold), "threshold must be finite");
  ResistTaps taps;
  std::string why;
  if (!resist_taps(sigma_nm, pixel_nm, &taps, &why)) {
    set_error("%s", why.c_str());
    return LITHO_EINVAL;
  }
  LITHO_REQUIRE(2 * taps.radius < n, "blur radius must be below n/2");
  ProfScope ps(kStageResist, static_cast<cudaStream_t>(stream), 1);
  LITHO_TRY_CUDA(launch_resist(intensity_dev, planes, n, taps, float(threshold), iblur_dev, printed_dev,
                               static_cast<cudaStream_t>(stream)));
  return LITHO_OK;
}

// ---- rectangle rasterisation -------------------------------------------------------------------

static bool raster_args_ok(int b, int n, int64_t max_rects, int max_side_px) {
  return b >= 1 && b <= 65535 && n >= 16 && n % 16 == 0 && n <= 65536 && max_rects >= 0 && max_side_px >= 1 &&
         max_side_px <= n && max_rects * raster_tiles_per_rect(max_side_px) < (int64_t(1) << 31);
}

litho_status litho_rasterize_workspace_size(int b, int n, int64_t max_rects, int max_side_px, size_t* bytes) {
  LITHO_REQUIRE(bytes, "null argument");
  LITHO_REQUIRE(raster_args_ok(b, n, max_rects, max_side_px),
                "need 1 <= b <= 65535, n a multiple of 16, 1 <= max_side_px <= n and a bounded tile list");
  *bytes = raster_workspace_bytes(b, n, max_rects, max_side_px);
  return LITHO_OK;
}

litho_status litho_rasterize(const float* rects_dev, const int64_t* rect_start_dev, int b, int64_t max_rects,
                             int max_side_px, int n, float* mask_dev, void* workspace_dev, size_t workspace_bytes,
                             void* stream) {
  LITHO_REQUIRE(rect_start_dev && mask_dev && workspace_dev && (rects_dev || max_rects == 0), "null argument");
  LITHO_REQUIRE(raster_args_ok(b, n, max_rects, max_side_px),
                "need 1 <= b <= 65535, n a multiple of 16, 1 <= max_side_px <= n and a bounded tile list");
  LITHO_REQUIRE((reinterpret_cast<uintptr_t>(rects_dev) & 15) == 0 && (reinterpret_cast<uintptr_t>(workspace_dev) & 255) == 0,
                "rects_dev must be 16-byte and workspace 256-byte aligned");
  const size_t need = raster_workspace_bytes(b, n, max_rects, max_side_px);
  if (workspace_bytes < need) {
    set_error("workspace too small: %zu bytes given, %zu needed", workspace_bytes, need);
    return LITHO_ENOMEM;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ProfScope ps(kStageRaster, st, 5);
  LITHO_TRY_CUDA(launch_raster(reinterpret_cast<const float4*>(rects_dev),
                               reinterpret_cast<const long long*>(rect_start_dev), b, max_rects, max_side_px, n,
                               mask_dev, workspace_dev, st));
  return LITHO_OK;
}

// ---- contours and edge placement ---------------------------------------------------------------

litho_status litho_contours_workspace_size(int planes, int n, size_t* bytes) {
  LITHO_REQUIRE(bytes && planes >= 1 && n >= 2, "bad argument");
  *bytes = contour_workspace_bytes(planes, n);
  return LITHO_OK;
}

litho_status litho_contours(const float* iblur_dev, int planes, int n, double threshold, float* seg_dev,
                            int32_t* cell_dev, int64_t capacity, int64_t* plane_start_dev, void* workspace_dev,
                            size_t workspace_bytes, void* stream) {
  LITHO_REQUIRE(iblur_dev && plane_start_dev && workspace_dev, "null argument");
  LITHO_REQUIRE(planes >= 1 && planes <= 65535 && n >= 2 && n <= 65536, "planes in [1, 65535] and n in [2, 65536] required");
  LITHO_REQUIRE(capacity >= 0 && (capacity == 0 || seg_dev), "seg_dev needed for a nonzero capacity");
  LITHO_REQUIRE(std::isfinite(threshold), "threshold must be finite");
  LITHO_REQUIRE((reinterpret_cast<uintptr_t>(seg_dev) & 15) == 0 && (reinterpret_cast<uintptr_t>(workspace_dev) & 255) == 0,
                "seg_dev must be 16-byte and workspace 256-byte aligned");
  if (workspace_bytes < contour_workspace_bytes(planes, n)) {
    set_error("workspace too small: %zu bytes given, %zu needed", workspace_bytes, contour_workspace_bytes(planes, n));
    return LITHO_ENOMEM;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ProfScope ps(kStageContours, st, 4);
  LITHO_TRY_CUDA(launch_contours(iblur_dev, planes, n, float(threshold), reinterpret_cast<float4*>(seg_dev), cell_dev,
                                 capacity, reinterpret_cast<long long*>(plane_start_dev), workspace_dev, st));
  return LITHO_OK;
}

litho_status litho_epe(const float* iblur_dev, int planes, int n, double pixel_nm, double threshold,
                       const float* points_dev, int m, float* epe_dev, void* stream) {
  LITHO_REQUIRE(iblur_dev && points_dev && epe_dev, "null argument");
  LITHO_REQUIRE(planes >= 1 && n >= 2 && m >= 0, "planes >= 1, n >= 2, m >= 0 required");
  LITHO_REQUIRE(pixel_nm > 0 && std::isfinite(threshold), "pixel_nm > 0 and a finite threshold required");
  LITHO_REQUIRE((reinterpret_cast<uintptr_t>(points_dev) & 7) == 0, "points_dev must be 8-byte aligned");
  if (m == 0) return LITHO_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ProfScope ps(kStageEpe, st, 1);
  LITHO_TRY_CUDA(launch_epe(iblur_dev, planes, n, float(pixel_nm), float(threshold),
                            reinterpret_cast<const float2*>(points_dev), m, epe_dev, st));
  return LITHO_OK;
}

litho_status litho_epe_batch(const float* iblur_dev, int clips, int planes, int n, double pixel_nm, double threshold,
                             const float* points_dev, const int64_t* start_dev, int64_t m_total, float* epe_dev,
                             void* stream) {
  LITHO_REQUIRE(iblur_dev && points_dev && start_dev && epe_dev, "null argument");
  LITHO_REQUIRE(clips >= 1 && planes >= 1 && n >= 2 && m_total >= 0, "clips >= 1, planes >= 1, n >= 2, m_total >= 0");
  LITHO_REQUIRE(pixel_nm > 0 && std::isfinite(threshold), "pixel_nm > 0 and a finite threshold required");
  LITHO_REQUIRE((reinterpret_cast<uintptr_t>(points_dev) & 7) == 0 && (reinterpret_cast<uintptr_t>(start_dev) & 7) == 0,
                "points_dev and start_dev must be 8-byte aligned");
  if (m_total == 0) return LITHO_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ProfScope ps(kStageEpe, st, 1);
  LITHO_TRY_CUDA(launch_epe_batch(iblur_dev, clips, planes, n, float(pixel_nm), float(threshold),
                                  reinterpret_cast<const float2*>(points_dev),
                                  reinterpret_cast<const long long*>(start_dev), m_total, epe_dev, st));
  return LITHO_OK;
}

litho_status litho_epe_through_focus(const float* epe_dev, int planes, int m, int f0, int fp, int fn, double tol_neg,
                                     double tol_pos, float* avg_dev, float* eff_dev, void* stream) {
  LITHO_REQUIRE(epe_dev && (avg_dev || eff_dev), "null argument");
  LITHO_REQUIRE(m >= 0 && f0 >= 0 && fp >= 0 && fn >= 0 && f0 < planes && fp < planes && fn < planes,
                "plane indices must lie in [0, planes)");
  LITHO_REQUIRE(tol_neg <= tol_pos, "tol_neg <= tol_pos required");
  if (m == 0) return LITHO_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ProfScope ps(kStageEpe, st, 1);
  LITHO_TRY_CUDA(launch_epe_focus(epe_dev, m, f0, fp, fn, float(tol_neg), float(tol_pos), avg_dev, eff_dev, st));
  return LITHO_OK;
}

}  // extern "C"
