// Host FP64 optics builder: source sampling, pupil, TCC eigen-kernels.
//
// Paper Section III.A, Eqs. (2)-(3).  TCC(f1, f2) = sum_s w_s P(f1 + s) P*(f2 + s)
// is A A^H with A[u, s] = sqrt(w_s) P(f_u + sigma_s f_NA).  Its nonzero eigenpairs
// follow from the Ns x Ns Gram matrix G = A^H A: G v = lam v gives the unit
// eigenvector Phi = A v / sqrt(lam) of A A^H with the same lam.  The dense TCC
// over the crop (up to 200k x 200k) is never formed.
//
// This is the only FP64 stage of the forward path; everything after it runs on
// the GPU.  The eigensolver is a cyclic complex Jacobi method (Hermitian
// version of Jacobi's 1846 rotation method: each rotation zeroes one
// off-diagonal pair after a phase change that makes it real).
#include <cmath>
#include <cstring>
#include <algorithm>
#include <thread>

#include "litho_internal.h"

namespace litho {

namespace {

// Inclusive lattice membership with a 1e-12 relative slack so boundary points count.
bool in_annulus(int i, int j, double h, double s_in, double s_out) {
  const double r2 = double(i) * i + double(j) * j;
  return r2 >= (s_in * h) * (s_in * h) * (1.0 - 1e-12) && r2 <= (s_out * h) * (s_out * h) * (1.0 + 1e-12);
}

bool in_quadrupole(int i, int j, double h, double c, double r) {
  const double cc = c * h, rr = (r * h) * (r * h) * (1.0 + 1e-12);
  const double centres[4][2] = {{cc, 0.0}, {-cc, 0.0}, {0.0, cc}, {0.0, -cc}};
  for (auto& p : centres) {
    const double dx = i - p[0], dy = j - p[1];
    if (dx * dx + dy * dy <= rr) return true;
  }
  return false;
}

cd pupil_value(double fx, double fy, double fna2, double kn, double z) {
  const double f2 = fx * fx + fy * fy;
  if (!(f2 <= fna2)) return cd(0.0, 0.0);
  if (z == 0.0) return cd(1.0, 0.0);
  const double kz = std::sqrt(std::max(kn * kn - f2, 0.0)) - kn;
  const double ph = 2.0 * M_PI * z * kz;
  return cd(std::cos(ph), std::sin(ph));
}

template <class F>
void parallel_for(long long count, F&& fn) {
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (count < 4096) nt = 1;
  std::vector<std::thread> th;
  const long long chunk = (count + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const long long lo = t * chunk, hi = std::min(count, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back([=, &fn] { fn(lo, hi, t); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

bool sample_source(const litho_optics& o, SourcePoints* out, std::string* why) {
  if (o.src_grid < 3 || (o.src_grid % 2) == 0) {
    *why = "src_grid must be odd and >= 3";
    return false;
  }
  const int h = (o.src_grid - 1) / 2;
  out->sx.clear();
  out->sy.clear();
  out->w.clear();
  double wsum = 0.0;
  for (int j = -h; j <= h; ++j) {
    for (int i = -h; i <= h; ++i) {
      double w = 0.0;
      if (o.kind == LITHO_SRC_ANNULAR) {
        w = in_annulus(i, j, h, o.sigma_in, o.sigma_out) ? 1.0 : 0.0;
      } else if (o.kind == LITHO_SRC_QUADRUPOLE) {
        w = in_quadrupole(i, j, h, o.pole_sigma, o.pole_radius) ? 1.0 : 0.0;
      } else if (o.kind == LITHO_SRC_CUSTOM) {
        if (!o.custom_w) {
          *why = "custom source without weights";
          return false;
        }
        w = o.custom_w[(j + h) * o.src_grid + (i + h)];
        if (w < 0.0 || !std::isfinite(w)) {
          *why = "custom source weights must be finite and >= 0";
          return false;
        }
      } else {
        *why = "unknown source kind";
        return false;
      }
      if (w > 0.0) {
        const double sx = double(i) / h, sy = double(j) / h;
        if (sx * sx + sy * sy > 1.0 + 1e-12) {
          *why = "source points must lie inside the pupil (|sigma| <= 1)";
          return false;
        }
        out->sx.push_back(sx);
        out->sy.push_back(sy);
        out->w.push_back(w);
        wsum += w;
      }
    }
  }
  if (out->w.empty() || !(wsum > 0.0)) {
    *why = "source has no points";
    return false;
  }
  for (double& w : out->w) w /= wsum;
  return true;
}

int band_crop(const litho_optics& o, const SourcePoints& s, int n, double pixel_nm) {
  double smax = 0.0;
  for (size_t i = 0; i < s.w.size(); ++i) smax = std::max(smax, std::sqrt(s.sx[i] * s.sx[i] + s.sy[i] * s.sy[i]));
  const double fb = (1.0 + smax) * o.na / o.wavelength_nm;
  const int rb = int(std::floor(fb * n * pixel_nm));
  int c = 2 * rb + 2;
  c = ((c + 31) / 32) * 32;
  return std::min(c, n);
}

void hermitian_jacobi(std::vector<cd>& a, int n, std::vector<double>& ev, std::vector<cd>& v) {
  v.assign(size_t(n) * n, cd(0.0, 0.0));
  for (int i = 0; i < n; ++i) v[size_t(i) * n + i] = 1.0;
  auto A = [&](int r, int c) -> cd& { return a[size_t(r) * n + c]; };
  double fro = 0.0;
  for (auto& x : a) fro += std::norm(x);
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += std::norm(A(p, q));
    if (std::sqrt(off) <= 1e-16 * fro) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const cd b = A(p, q);
        const double ab = std::abs(b);
        if (ab <= 1e-300 || ab <= 1e-18 * fro) {
          A(p, q) = A(q, p) = 0.0;
          continue;
        }
        // phase e^{i phi} = b/|b| makes the pair real; then a real rotation
        // with tan(theta) = t, t the smaller root of t^2 + 2 zeta t - 1 = 0.
        const cd ph = b / ab;
        const double app = A(p, p).real(), aqq = A(q, q).real();
        const double zeta = (aqq - app) / (2.0 * ab);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        // U restricted to (p, q): [[c, s], [-s conj(ph), c conj(ph)]]
        const cd upp = c, upq = s, uqp = -s * std::conj(ph), uqq = c * std::conj(ph);
        for (int r = 0; r < n; ++r) {  // A <- A U
          const cd x = A(r, p), y = A(r, q);
          A(r, p) = x * upp + y * uqp;
          A(r, q) = x * upq + y * uqq;
        }
        for (int r = 0; r < n; ++r) {  // A <- U^H A
          const cd x = A(p, r), y = A(q, r);
          A(p, r) = std::conj(upp) * x + std::conj(uqp) * y;
          A(q, r) = std::conj(upq) * x + std::conj(uqq) * y;
        }
        A(p, q) = A(q, p) = 0.0;
        A(p, p) = A(p, p).real();
        A(q, q) = A(q, q).real();
        for (int r = 0; r < n; ++r) {  // V <- V U
          const cd x = v[size_t(r) * n + p], y = v[size_t(r) * n + q];
          v[size_t(r) * n + p] = x * upp + y * uqp;
          v[size_t(r) * n + q] = x * upq + y * uqq;
        }
      }
    }
  }
  ev.resize(n);
  for (int i = 0; i < n; ++i) ev[i] = A(i, i).real();
}

bool build_focus_kernels(const litho_optics& o, const SourcePoints& s, int n, double pixel_nm, double z_nm, int k,
                         int crop, FocusKernels* out, std::string* why) {
  const int ns = int(s.w.size());
  const long long nb = (long long)crop * crop;
  const double fna = o.na / o.wavelength_nm, fna2 = fna * fna, kn = o.n_medium / o.wavelength_nm;
  // A[u][s], u over the crop in [v][u] order
  std::vector<cd> amat(size_t(nb) * ns);
  parallel_for(nb, [&](long long lo, long long hi, unsigned) {
    for (long long b = lo; b < hi; ++b) {
      const int cv = int(b / crop), cu = int(b % crop);
      const double fy = double(cv - crop / 2) / (n * pixel_nm), fx = double(cu - crop / 2) / (n * pixel_nm);
      for (int j = 0; j < ns; ++j) {
        amat[size_t(b) * ns + j] =
            std::sqrt(s.w[j]) * pupil_value(fx + s.sx[j] * fna, fy + s.sy[j] * fna, fna2, kn, z_nm);
      }
    }
  });
  // G = A^H A, accumulated per thread then summed
  const unsigned max_t = 16;
  std::vector<std::vector<cd>> part(max_t, std::vector<cd>(size_t(ns) * ns, cd(0, 0)));
  parallel_for(nb, [&](long long lo, long long hi, unsigned t) {
    auto& g = part[t];
    for (long long b = lo; b < hi; ++b) {
      const cd* row = &amat[size_t(b) * ns];
      bool any = false;
      for (int j = 0; j < ns; ++j) any |= (row[j] != cd(0, 0));
      if (!any) continue;
      for (int p = 0; p < ns; ++p) {
        const cd cp = std::conj(row[p]);
        if (cp == cd(0, 0)) continue;
        cd* gp = &g[size_t(p) * ns];
        for (int q = 0; q < ns; ++q) gp[q] += cp * row[q];
      }
    }
  });
  std::vector<cd> g(size_t(ns) * ns, cd(0, 0));
  for (auto& pp : part)
    for (size_t i = 0; i < g.size(); ++i) g[i] += pp[i];
  for (int p = 0; p < ns; ++p)  // exact Hermitian symmetry
    for (int q = p + 1; q < ns; ++q) {
      const cd avg = 0.5 * (g[size_t(p) * ns + q] + std::conj(g[size_t(q) * ns + p]));
      g[size_t(p) * ns + q] = avg;
      g[size_t(q) * ns + p] = std::conj(avg);
    }
  double trace = 0.0;
  for (int p = 0; p < ns; ++p) trace += g[size_t(p) * ns + p].real();

  std::vector<double> ev;
  std::vector<cd> vec;
  hermitian_jacobi(g, ns, ev, vec);
  std::vector<int> order(ns);
  for (int i = 0; i < ns; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] > ev[b]; });
  const double top = ev[order[0]];
  out->lambda.assign(k, 0.0);
  out->phi.assign(size_t(k) * nb, cd(0, 0));
  out->trace = trace;
  out->rank = 0;
  for (int i = 0; i < ns; ++i)
    if (ev[order[i]] > 1e-12 * top) out->rank++;
  auto lam_at = [&](int i) { return i < ns ? std::max(ev[order[i]], 0.0) : 0.0; };
  out->gap = (k >= 1) ? lam_at(k - 1) - lam_at(k) : 0.0;
  const int kk = std::min(k, out->rank);
  for (int i = 0; i < kk; ++i) out->lambda[i] = ev[order[i]];
  parallel_for(nb, [&](long long lo, long long hi, unsigned) {
    for (int i = 0; i < kk; ++i) {
      const int col = order[i];
      const double inv = 1.0 / std::sqrt(out->lambda[i]);
      for (long long b = lo; b < hi; ++b) {
        const cd* row = &amat[size_t(b) * ns];
        cd acc(0, 0);
        for (int j = 0; j < ns; ++j) acc += row[j] * vec[size_t(j) * ns + col];
        out->phi[size_t(i) * nb + b] = acc * inv;
      }
    }
  });
  (void)why;
  return true;
}

}  // namespace litho
