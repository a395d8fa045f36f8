// Host side of libgfh: grid derivation (Sec. VI), fixed-point tables, column tables, contexts and
// plans.  Compiled with -ffp-contract=off so that every double expression rounds exactly as
// written (no fused multiply-add), which the bit-exact tables rely on.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>

#include "gfh_internal.h"

namespace {

int64_t fixed_floor(double v) { return (int64_t)std::floor(std::ldexp(v, GFH_FRAC_BITS)); }

int64_t floor_shift(int64_t v) { return v >> GFH_FRAC_BITS; }  // arithmetic shift = floor

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// n = 0 selects the original FrequencyHough (Sec. III Eq. fdotslope): x = -f, x0 = -f0 and
// x0 = x - k t with k = -fdot, the orientation and slope convention of Eq. transform's
// x0 = x - (n-1) k t with (n-1) replaced by 1.  Only this form accepts k < 0 (spin-up).
bool original_fh(const gfh_grid* g) { return g->n == 0.0; }

double slope_of(const gfh_grid* g) { return original_fh(g) ? 1.0 : g->n - 1.0; }

// x of frequency f: Eq. transform (n > 1) or -f (n = 0).
double x_of_f(const gfh_grid* g, double f) {
  return original_fh(g) ? -f : std::pow(f, 1.0 - g->n);
}

bool grid_request_ok(const gfh_grid* g) {
  return g && (g->n > 1.0 || g->n == 0.0) && g->df > 0.0 && g->bin_lo >= 1 &&
         g->bin_hi >= g->bin_lo && g->n_fft >= 1 && g->n_k >= 1 && g->t_first >= 0.0 &&
         g->t_hop >= 0.0 && g->t_obs > 0.0 && (g->k_min >= 0.0 || g->n == 0.0) &&
         std::isfinite(g->k_min) && g->ana_hi > g->ana_lo && g->band_hz > 0.0 &&
         std::isfinite(g->n) && std::isfinite(g->df);
}

bool grid_made(const gfh_grid* g) {
  return grid_request_ok(g) && g->dx0 > 0.0 && g->dk > 0.0 && g->n_x0 > 0 &&
         g->ld_x0 >= g->n_x0 && g->n_bands > 0;
}

}  // namespace

extern "C" const char* gfh_strerror(int code) {
  switch (code) {
    case GFH_OK: return "ok";
    case GFH_ERR_ARG: return "invalid argument";
    case GFH_ERR_SIZE: return "size out of range or capacity too small";
    case GFH_ERR_CUDA: return "CUDA or cuFFT call failed";
    case GFH_ERR_INPUT: return "device-side input check failed (unsorted peaks or index out of range)";
    case GFH_ERR_TIMEOUT: return "bounded device-side wait ran out";
    case GFH_ERR_NOMEM: return "allocation failed";
    default: return "unknown error";
  }
}

// ---- Sec. VI grids ----------------------------------------------------------------------------

extern "C" int gfh_grid_make(gfh_grid* g) {
  if (!grid_request_ok(g)) return GFH_ERR_ARG;
  const double n = g->n;
  const double m = slope_of(g);
  if (!(g->f_max > 0.0)) g->f_max = (double)g->bin_hi * g->df;
  g->dx0 = m * g->df / std::pow(g->f_max, n);                        // Sec. VI.C (df for n = 0)
  if (!(g->dk > 0.0)) g->dk = g->dx0 / (m * g->t_obs);
  const double k_max = g->k_min + (double)(g->n_k - 1) * g->dk;
  const double t_max = g->t_first + (double)(g->n_fft - 1) * g->t_hop;
  const double x_top = x_of_f(g, ((double)g->bin_hi + 0.5) * g->df);  // Eq. transform
  const double x_bot = x_of_f(g, ((double)g->bin_lo - 0.5) * g->df);
  // lowest x0 of any line: x_top moved by the largest positive k; highest: x_bot moved by the most
  // negative k (none for k_min >= 0)
  g->x0_min = x_top - m * (k_max > 0.0 ? k_max : 0.0) * t_max - g->dx0;
  const double x0_hi = g->k_min < 0.0 ? x_bot - m * g->k_min * t_max : x_bot;
  const double w = std::ceil((x0_hi - g->x0_min) / g->dx0);
  if (!(g->dx0 > 0.0) || !std::isfinite(w) || w < 0.0 || w > 2.0e9) return GFH_ERR_SIZE;
  g->n_x0 = (int64_t)w + 1;
  g->ld_x0 = (g->n_x0 + 31) / 32 * 32;
  const double nb = std::ceil((g->ana_hi - g->ana_lo) / g->band_hz);
  if (!(nb >= 1.0) || nb > 1.0e8) return GFH_ERR_ARG;
  g->n_bands = (int32_t)nb;
  return GFH_OK;
}

int gfh_host_tables(const gfh_grid* g, std::vector<int64_t>& U, std::vector<int64_t>& B,
                    std::vector<int64_t>& S) {
  if (!grid_made(g)) return GFH_ERR_ARG;
  const int J = g->bin_hi - g->bin_lo + 1;
  U.resize((size_t)J + 1);
  for (int e = 0; e <= J; ++e) {
    const double f = ((double)(g->bin_lo + e) - 0.5) * g->df;
    const double x = x_of_f(g, f);
    U[e] = fixed_floor((x - g->x0_min) / g->dx0);
  }
  B.resize(g->n_fft);
  S.resize(g->n_fft);
  const double m = slope_of(g);
  for (int i = 0; i < g->n_fft; ++i) {
    const double t = g->t_first + (double)i * g->t_hop;
    B[i] = fixed_floor(m * g->k_min * t / g->dx0);
    S[i] = fixed_floor(m * g->dk * t / g->dx0);
  }
  return GFH_OK;
}

int gfh_host_columns(const gfh_grid* g, std::vector<int32_t>& band, std::vector<double>& f0,
                     std::vector<double>& f0n) {
  if (!grid_made(g)) return GFH_ERR_ARG;
  const int64_t W = g->n_x0;
  band.assign((size_t)g->ld_x0, -1);
  f0.assign((size_t)W, 0.0);
  f0n.assign((size_t)W, 0.0);
  const double e = -1.0 / (g->n - 1.0);
  for (int64_t m = 0; m < W; ++m) {
    const double x0c = g->x0_min + ((double)m + 0.5) * g->dx0;
    const double f = original_fh(g) ? -x0c : (x0c > 0.0 ? std::pow(x0c, e) : 0.0);
    if (!(f > 0.0)) continue;
    f0[m] = f;
    f0n[m] = std::pow(f, g->n);
    if (g->ana_lo <= f && f < g->ana_hi) {
      int32_t b = (int32_t)std::floor((f - g->ana_lo) / g->band_hz);
      if (b > g->n_bands - 1) b = g->n_bands - 1;
      band[m] = b;
    }
  }
  return GFH_OK;
}

extern "C" int gfh_grid_tables(const gfh_grid* g, int64_t* h_U, int64_t* h_B, int64_t* h_S) {
  std::vector<int64_t> U, B, S;
  int rc = gfh_host_tables(g, U, B, S);
  if (rc) return rc;
  if (h_U) std::memcpy(h_U, U.data(), U.size() * sizeof(int64_t));
  if (h_B) std::memcpy(h_B, B.data(), B.size() * sizeof(int64_t));
  if (h_S) std::memcpy(h_S, S.data(), S.size() * sizeof(int64_t));
  return GFH_OK;
}

extern "C" int gfh_grid_columns(const gfh_grid* g, int32_t* h_band, double* h_f0, double* h_f0n) {
  std::vector<int32_t> band;
  std::vector<double> f0, f0n;
  int rc = gfh_host_columns(g, band, f0, f0n);
  if (rc) return rc;
  if (h_band) std::memcpy(h_band, band.data(), (size_t)g->n_x0 * sizeof(int32_t));
  if (h_f0) std::memcpy(h_f0, f0.data(), f0.size() * sizeof(double));
  if (h_f0n) std::memcpy(h_f0n, f0n.data(), f0n.size() * sizeof(double));
  return GFH_OK;
}

// ---- contexts -----------------------------------------------------------------------------------

extern "C" int gfh_create(gfh_ctx** out, int device, void* stream) {
  if (!out) return GFH_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return GFH_ERR_CUDA;
  GFH_CUDA_TRY(cudaSetDevice(device));
  gfh_ctx* c = new (std::nothrow) gfh_ctx();
  if (!c) return GFH_ERR_NOMEM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&c->d_flag, sizeof(unsigned int)) != cudaSuccess ||
      cudaMemset(c->d_flag, 0, sizeof(unsigned int)) != cudaSuccess ||
      cudaMallocHost(&c->h_pinned, 64) != cudaSuccess) {
    gfh_destroy(c);
    return GFH_ERR_CUDA;
  }
  // image channel 0 for small peak counts: bf16 (round to nearest even) of float(log1p(count))
  std::vector<uint16_t> tab(kLogTable);
  for (int i = 0; i < kLogTable; ++i) {
    const float f = (float)std::log1p((double)i);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    tab[i] = (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
  }
  if (cudaMalloc(&c->d_log1p, kLogTable * sizeof(uint16_t)) != cudaSuccess ||
      cudaMemcpy(c->d_log1p, tab.data(), kLogTable * sizeof(uint16_t), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    gfh_destroy(c);
    return GFH_ERR_CUDA;
  }
  *out = c;
  return GFH_OK;
}

extern "C" int gfh_destroy(gfh_ctx* c) {
  if (!c) return GFH_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& f : c->fft)
    if (f.valid) cufftDestroy(f.h);
  if (c->pm_buf) cudaFree(c->pm_buf);
  if (c->d_flag) cudaFree(c->d_flag);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->d_log1p) cudaFree(c->d_log1p);
  delete c;
  return GFH_OK;
}

extern "C" int gfh_set_stream(gfh_ctx* c, void* stream) {
  if (!c) return GFH_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  for (auto& f : c->fft)
    if (f.valid && cufftSetStream(f.h, c->stream) != CUFFT_SUCCESS) return GFH_ERR_CUDA;
  return GFH_OK;
}

extern "C" int gfh_check(gfh_ctx* c) {
  if (!c) return GFH_ERR_ARG;
  GFH_CUDA_TRY(cudaSetDevice(c->device));
  unsigned int flag = 0;
  GFH_CUDA_TRY(cudaMemcpyAsync(&flag, c->d_flag, sizeof(flag), cudaMemcpyDeviceToHost, c->stream));
  GFH_CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (flag) {
    GFH_CUDA_TRY(cudaMemsetAsync(c->d_flag, 0, sizeof(unsigned int), c->stream));
    GFH_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (flag & GFH_FLAG_TIMEOUT) return GFH_ERR_TIMEOUT;
    return (flag & (GFH_FLAG_UNSORTED | GFH_FLAG_FFT_RANGE)) ? GFH_ERR_INPUT : GFH_ERR_SIZE;
  }
  return GFH_OK;
}

// ---- grids on n and k (Sec. VI) -------------------------------------------------------------------

namespace {

// f(t) / f0 of Eq. powlaws at u = |fdot0| t / f0.
double powlaw_ratio(double n, double u) { return std::exp(-std::log1p((n - 1.0) * u) / (n - 1.0)); }

// Largest |f_{n2} - f_{n1}| over the f0 and u lattice of gfh_n_grid.
double dn_max_df(double n1, double n2, double f_min, double f_max, double fdot_hi, double t_obs) {
  constexpr int kF = 64, kU = 256;
  double best = 0.0;
  for (int a = 0; a < kF; ++a) {
    const double f0 = f_min * std::pow(f_max / f_min, (double)a / (kF - 1));
    const double umax = fdot_hi * t_obs / f0;
    for (int b = 0; b < kU; ++b) {
      const double u = umax * b / (kU - 1);
      const double d = f0 * std::fabs(powlaw_ratio(n2, u) - powlaw_ratio(n1, u));
      if (d > best) best = d;
    }
  }
  return best;
}

}  // namespace

extern "C" int gfh_n_grid(double n_lo, double n_hi, double df, double f_min, double f_max,
                          double fdot_hi, double t_obs, int32_t cap, double* h_n, int32_t* n_out) {
  if (!h_n || !n_out || cap < 1 || !(n_lo > 1.0) || !(n_hi >= n_lo) || !(df > 0.0) ||
      !(f_min > 0.0) || !(f_max >= f_min) || !(fdot_hi >= 0.0) || !(t_obs > 0.0))
    return GFH_ERR_ARG;
  int32_t cnt = 0;
  h_n[cnt++] = n_lo;
  double n = n_lo;
  while (n < n_hi) {
    if (cnt >= cap) { *n_out = cnt; return GFH_ERR_SIZE; }
    const double span = n_hi - n;
    if (dn_max_df(n, n + span, f_min, f_max, fdot_hi, t_obs) <= df) {
      h_n[cnt++] = n_hi;
      break;
    }
    double lo = 0.0, hi = span;
    while (hi - lo > 1e-9 * hi) {
      const double mid = 0.5 * (lo + hi);
      if (dn_max_df(n, n + mid, f_min, f_max, fdot_hi, t_obs) <= df) lo = mid;
      else hi = mid;
    }
    if (lo <= 0.0) { *n_out = cnt; return GFH_ERR_ARG; }
    n = n + lo;
    h_n[cnt++] = n;
  }
  *n_out = cnt;
  return GFH_OK;
}

extern "C" int gfh_k_segments(double n, double df, double f_min, double f_max, double fdot_lo,
                              double fdot_hi, double growth, int32_t max_rows, int32_t cap,
                              gfh_k_segment* h_out, int32_t* n_out) {
  if (!h_out || !n_out || cap < 1 || !(n > 1.0) || !(df > 0.0) || !(f_min > 0.0) ||
      !(f_max >= f_min) || !(fdot_lo > 0.0) || !(fdot_hi >= fdot_lo) || !(growth >= 1.0) ||
      max_rows < 1)
    return GFH_ERR_ARG;
  const double c = 1.0 - std::pow(1.0 + df / f_max, -n);
  const double k_lo = fdot_lo / std::pow(f_max, n), k_hi = fdot_hi / std::pow(f_min, n);
  const double full = std::floor((growth - 1.0) / c) + 1.0;
  const int32_t rows_full = full > (double)max_rows ? max_rows : (int32_t)full;
  int32_t cnt = 0;
  double k = k_lo;
  for (;;) {
    if (cnt >= cap) { *n_out = cnt; return GFH_ERR_SIZE; }
    const double dk = k * c;
    int32_t rows = rows_full;
    if (k < k_hi) {
      const double need = std::ceil((k_hi - k) / dk) + 1.0;
      if (need < (double)rows) rows = (int32_t)need;
    } else {
      rows = 1;
    }
    if (rows < 1) rows = 1;
    h_out[cnt].k_min = k;
    h_out[cnt].dk = dk;
    h_out[cnt].n_k = rows;
    h_out[cnt].reserved = 0;
    ++cnt;
    if (k + (rows - 1) * dk >= k_hi) break;
    k = k + rows * dk;
  }
  *n_out = cnt;
  return GFH_OK;
}

// ---- Sec. VI.D: longer FFTs for later times ---------------------------------------------------

namespace {

// First time at which the largest |fdot(t)| over the power laws of braking index n with
// f0 <= f_hi and |fdot0| <= fdot_hi falls to fdot.  A member's |fdot(t)| = fdot0 (1 + u)^(-n/(n-1)),
// u = (n-1) fdot0 t / f0, peaks over fdot0 at u = n-1: the bound is the fastest member's while
// t fdot_hi < f_hi and f_hi n^(-n/(n-1)) / t after that.
double time_of_spindown(double fdot, double n, double f_hi, double fdot_hi) {
  if (fdot_hi <= fdot) return 0.0;
  const double t1 = (std::pow(fdot_hi / fdot, (n - 1.0) / n) - 1.0) * f_hi / ((n - 1.0) * fdot_hi);
  if (t1 * fdot_hi < f_hi) return t1;
  return f_hi * std::pow(n, -n / (n - 1.0)) / fdot;
}

}  // namespace

extern "C" int gfh_tfft_portions(double n, double f_hi, double fdot_hi, double t_fft0,
                                 double t_obs, int32_t max_levels, int32_t cap,
                                 gfh_portion* h_out, int32_t* n_out) {
  if (!h_out || !n_out || cap < 1 || !(n > 1.0) || !std::isfinite(n) || !(f_hi > 0.0) ||
      !(fdot_hi > 0.0) || !(t_fft0 > 0.0) || !(t_obs > 0.0) || max_levels < 1 || max_levels > 30)
    return GFH_ERR_ARG;
  int32_t cnt = 0;
  for (int L = 0; L < max_levels; ++L) {
    const double T = t_fft0 * std::ldexp(1.0, L);                    // Eq. dot_tfft: fdot <= 1/T^2
    double a = time_of_spindown(1.0 / (T * T), n, f_hi, fdot_hi);
    if (a > t_obs) a = t_obs;
    double b = t_obs;
    if (L + 1 < max_levels) {
      b = time_of_spindown(1.0 / ((2.0 * T) * (2.0 * T)), n, f_hi, fdot_hi);
      if (b > t_obs) b = t_obs;
    }
    if (b - a >= T) {
      if (cnt >= cap) { *n_out = cnt; return GFH_ERR_SIZE; }
      h_out[cnt].level = L;
      h_out[cnt].reserved = 0;
      h_out[cnt].t_begin = a;
      h_out[cnt].t_end = b;
      h_out[cnt].t_fft = T;
      ++cnt;
    }
  }
  *n_out = cnt;
  return GFH_OK;
}

// ---- plans --------------------------------------------------------------------------------------

namespace {

struct HostMap {
  std::vector<int64_t> U, B, S;
  std::vector<int32_t> band;
  std::vector<double> f0, f0n;
  int64_t cells = 0;
};

// Bin range [ja, jb] of the peaks that can touch columns [c0, c1) on rows [r0, r1) (tile planning).
// For bin j (local jl) and shift s in [s_min, s_max]: lo >= (U[jl+1]-s_max)>>32 and
// hi <= (U[jl]-s_min-1)>>32; U decreases with jl, so both conditions select a contiguous range.
void tile_bins(const gfh_grid& g, const HostMap& hm, int64_t s_min, int64_t s_max, int64_t c0,
               int64_t c1, int32_t* ja, int32_t* jb) {
  const int J = g.bin_hi - g.bin_lo + 1;
  if (c0 > g.n_x0 - 1) { *ja = 1; *jb = 0; return; }
  // smallest jl with floor((U[jl+1]-s_max)) <= c1-1
  int lo = 0, hi = J;  // answer in [0, J]; J means none
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (floor_shift(hm.U[mid + 1] - s_max) <= c1 - 1) hi = mid; else lo = mid + 1;
  }
  const int a = lo;
  // largest jl with floor((U[jl]-s_min-1)) >= c0
  lo = -1; hi = J - 1;  // answer in [-1, J-1]
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (floor_shift(hm.U[mid] - s_min - 1) >= c0) lo = mid; else hi = mid - 1;
  }
  const int b = lo;
  *ja = g.bin_lo + a;
  *jb = g.bin_lo + b;
}

// Bins per tile of the coarse-tile search's FFT sub-ranges (8 bytes each in shared memory) that
// fit beside a tile of `base` bytes without lowering the blocks per SM (228 KB per SM, 1 KB of it
// reserved per block, at most the Hough kernels' limit per block), at most 1024.
int sub_capacity(size_t base, int threads) {
  constexpr size_t kSmemSM = 228 * 1024, kReserve = 1024, kOwn = kMaxSmemBytes - kHoughSmemLimit;
  const int blocks = (int)std::min<size_t>(kSmemSM / (base + kOwn + kReserve), (size_t)(2048 / threads));
  if (blocks < 1) return 0;
  const size_t room = std::min(kSmemSM / blocks - kReserve - kOwn, kHoughSmemLimit);
  if (room <= base + 16) return 0;
  const size_t cap = std::min<size_t>((room - base - 16) / 8, 1024);
  return cap >= 32 ? (int)cap : 0;
}

// Number of FFTs whose interval of bin jl (local) meets columns c0 .. ub on some of the R rows
// from row0 (B_i + r S_i does not fall as i grows when k_min >= 0: two bisections).
int64_t window_ffts(const gfh_grid& g, const HostMap& hm, int jl, int row0, int R, int64_t c0,
                    int64_t ub) {
  const int64_t x_hi = hm.U[jl] - 1 - (c0 << GFH_FRAC_BITS);
  const int64_t y_lo = hm.U[jl + 1] - ((ub + 1) << GFH_FRAC_BITS);
  const int64_t r_last = (int64_t)row0 + R - 1;
  int lo = 0, hi = g.n_fft;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (hm.B[mid] + (int64_t)row0 * hm.S[mid] <= x_hi) lo = mid + 1; else hi = mid;
  }
  const int last = lo - 1;
  lo = 0;
  hi = last + 1;
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (hm.B[mid] + r_last * hm.S[mid] > y_lo) hi = mid; else lo = mid + 1;
  }
  return last - lo + 1;
}

// Whether a tile of the coarse-tile search walks only its bins' FFT sub-ranges: they fit
// (sub_cap), the shifts grow with the FFT (k_min >= 0) and, over up to 8 bins sampled across the
// tile's bin range, at most half the (FFT, bin) pairs read meet the tile.
bool tile_walks_sub_ranges(const gfh_grid& g, const HostMap& hm, const TileDev& t, int R,
                           int sub_cap) {
  const int nb = t.bin_b - t.bin_a + 1;
  if (sub_cap <= 0 || nb <= 0 || nb > sub_cap || g.k_min < 0.0 || g.n_fft < 1) return false;
  const int64_t c0 = t.col0;
  const int64_t ub = std::min<int64_t>(c0 + t.ncols - 1, g.n_x0 - 1);
  const int samples = std::min(nb, 8);
  int64_t meet = 0;
  for (int q = 0; q < samples; ++q) {
    const int jl = t.bin_a - g.bin_lo + (int)((int64_t)q * (nb - 1) / std::max(1, samples - 1));
    meet += std::max<int64_t>(0, window_ffts(g, hm, jl, t.row0, R, c0, ub));
  }
  return (double)meet <= 0.5 * (double)samples * (double)g.n_fft;
}

// Tiles of map m covering rows [r0, r1) x columns [c_lo, c_hi) (c_lo, c_hi multiples of 4) with
// the plan's tile shape; appended to `tiles`.
void map_tiles(const gfh_grid& g, const HostMap& hm, int m, const gfh_tile_config& tc, int r0,
               int r1, int64_t c_lo, int64_t c_hi, std::vector<TileDev>& tiles, int& max_bands) {
  for (int rr = r0; rr < r1; rr += tc.rows) {
    const int nr = std::min(tc.rows, r1 - rr);
    // With k_min >= 0, B and S are non-decreasing in i (dk > 0, t_i non-decreasing), so the
    // smallest shift of the row block is at (i = 0, rr) and the largest at (last i, last row).
    // With k_min < 0 (n = 0 only) B falls with i: the shift of FFT i is linear in the row, so
    // its extremes over the block are at the block's first and last rows, taken over every i.
    int64_t s_min = hm.B[0] + (int64_t)rr * hm.S[0];
    int64_t s_max = hm.B[g.n_fft - 1] + (int64_t)(rr + nr - 1) * hm.S[g.n_fft - 1];
    if (g.k_min < 0.0) {
      for (int i = 0; i < g.n_fft; ++i) {
        const int64_t a = hm.B[i] + (int64_t)rr * hm.S[i];
        const int64_t b = hm.B[i] + (int64_t)(rr + nr - 1) * hm.S[i];
        s_min = std::min(s_min, std::min(a, b));
        s_max = std::max(s_max, std::max(a, b));
      }
    }
    for (int64_t c0 = c_lo; c0 < c_hi; c0 += tc.cols) {
      TileDev t{};
      t.map = m;
      t.row0 = rr;
      t.nrows = nr;
      t.col0 = c0;
      t.ncols = (int32_t)std::min<int64_t>(tc.cols, c_hi - c0);
      tile_bins(g, hm, s_min, s_max, c0, c0 + t.ncols, &t.bin_a, &t.bin_b);
      t.band_lo = INT32_MAX;
      t.band_hi = -1;
      for (int64_t c = c0; c < c0 + t.ncols; ++c) {
        const int32_t b = hm.band[c];
        if (b >= 0) { t.band_lo = std::min(t.band_lo, b); t.band_hi = std::max(t.band_hi, b); }
      }
      if (t.band_hi < 0) t.band_lo = 0;
      else max_bands = std::max(max_bands, t.band_hi - t.band_lo + 1);
      tiles.push_back(t);
    }
  }
}

}  // namespace

extern "C" int gfh_plan_destroy(gfh_plan* p) {
  if (!p) return GFH_OK;
  if (p->ctx) {
    cudaSetDevice(p->ctx->device);
    if (p->ctx->stream) cudaStreamSynchronize(p->ctx->stream);
  }
  if (p->d_buf) cudaFree(p->d_buf);
  if (p->d_coarse_buf) cudaFree(p->d_coarse_buf);
  delete p;
  return GFH_OK;
}

extern "C" int gfh_plan_create(gfh_ctx* ctx, int32_t n_maps, const gfh_grid* grids,
                               int32_t* const* h_maps, gfh_candidate* const* h_cands,
                               gfh_map_stats* d_stats, const gfh_tile_config* cfg,
                               gfh_plan** out) {
  if (!ctx || !out || n_maps < 1 || !grids || !h_maps) return GFH_ERR_ARG;
  *out = nullptr;
  gfh_tile_config tc{16, 3072, 512, 0};
  if (cfg) {
    if (cfg->rows) tc.rows = cfg->rows;
    if (cfg->cols) tc.cols = cfg->cols;
    if (cfg->threads) tc.threads = cfg->threads;
    tc.form = cfg->form;
  }
  if (!(tc.rows == 4 || tc.rows == 8 || tc.rows == 16 || tc.rows == 32) || tc.cols < 128 || tc.cols % 128 ||
      tc.cols > 4096 || !(tc.form == 0 || tc.form == 1) ||
      !(tc.threads == 256 || tc.threads == 512 || (tc.threads == 1024 && tc.rows >= 16)))
    return GFH_ERR_ARG;
  const int nwarps = tc.threads / 32;
  if ((tc.cols / 128 + nwarps - 1) / nwarps > 4) return GFH_ERR_ARG;  // <= 4 chunks per warp

  std::vector<HostMap> hms(n_maps);
  std::vector<TileDev> tiles, tiles_x;
  std::vector<char> map_xd(n_maps, 0);
  int max_tile_bands = 1;
  size_t csr_entries = 0;
  for (int m = 0; m < n_maps; ++m) {
    const gfh_grid& g = grids[m];
    if (!grid_made(&g) || !h_maps[m]) return GFH_ERR_ARG;
    if ((double)g.n_k * (double)g.n_x0 >= 4294967295.0) return GFH_ERR_SIZE;
    if (h_cands && !h_cands[m]) return GFH_ERR_ARG;
    HostMap& hm = hms[m];
    int rc = gfh_host_tables(&g, hm.U, hm.B, hm.S);
    if (rc) return rc;
    rc = gfh_host_columns(&g, hm.band, hm.f0, hm.f0n);
    if (rc) return rc;
    int64_t ana_cols = 0;
    for (int64_t c = 0; c < g.n_x0; ++c) ana_cols += hm.band[c] >= 0;
    hm.cells = ana_cols * g.n_k;
    csr_entries += (size_t)(g.bin_hi - g.bin_lo + 2);
    if (((uintptr_t)h_maps[m]) % 16) return GFH_ERR_ARG;  // 16-byte vector stores
    // A line moving more than two columns per k row (coarse k steps, e.g. Eq. dkeqn's) costs
    // fewer events differenced along x0 on every row (2 per row) than along k (the columns it
    // crosses): such maps use the x-direction form.
    map_xd[m] = hm.S[g.n_fft - 1] > (int64_t(2) << GFH_FRAC_BITS);
    map_tiles(g, hm, m, tc, 0, g.n_k, 0, g.ld_x0, map_xd[m] ? tiles_x : tiles, max_tile_bands);
  }
  // The tile must fit in shared memory (layout of k_hough: tile, chunk sums, band keys).
  const bool select = h_cands != nullptr || d_stats != nullptr;
  const size_t smem = (size_t)tc.rows * (tc.cols + 2) * 4 + 32 * 4 * (tiles_x.empty() ? 1 : tc.rows) +
                      (select ? (size_t)max_tile_bands * 8 : 0);
  if (smem > kHoughSmemLimit) return GFH_ERR_SIZE;
  // Longest work first: bins x rows; the x-direction tiles form a second list after the others.
  auto by_work = [](const TileDev& a, const TileDev& b) {
    const int64_t wa = (int64_t)std::max(0, a.bin_b - a.bin_a + 1) * a.nrows;
    const int64_t wb = (int64_t)std::max(0, b.bin_b - b.bin_a + 1) * b.nrows;
    return wa > wb;
  };
  std::stable_sort(tiles.begin(), tiles.end(), by_work);
  std::stable_sort(tiles_x.begin(), tiles_x.end(), by_work);
  const int n_tiles_k = (int)tiles.size();
  tiles.insert(tiles.end(), tiles_x.begin(), tiles_x.end());

  // One device buffer: map descriptors | tiles | csr map index | keys | per-map tables.
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_maps = take(sizeof(MapDev) * n_maps);
  const size_t o_tiles = take(sizeof(TileDev) * tiles.size());
  const size_t o_csrmap = take(sizeof(int32_t) * csr_entries);
  size_t key_words = 0;
  for (int m = 0; m < n_maps; ++m) key_words += grids[m].n_bands + 2;
  const size_t o_keys = take(sizeof(unsigned long long) * key_words);
  std::vector<size_t> o_U(n_maps), o_B(n_maps), o_S(n_maps), o_band(n_maps), o_f0(n_maps),
      o_f0n(n_maps), o_csr(n_maps);
  for (int m = 0; m < n_maps; ++m) {
    o_U[m] = take(2 * sizeof(int64_t) * (hms[m].U.size() - 1));
    o_B[m] = take(2 * sizeof(int64_t) * hms[m].B.size());
    o_S[m] = 0;
    o_band[m] = take(sizeof(int32_t) * hms[m].band.size());
    o_f0[m] = take(sizeof(double) * hms[m].f0.size());
    o_f0n[m] = take(sizeof(double) * hms[m].f0n.size());
    o_csr[m] = take(sizeof(int64_t) * (size_t)(grids[m].bin_hi - grids[m].bin_lo + 2));
  }
  const size_t o_single = take(sizeof(int64_t) * 2);
  const size_t o_next = take(sizeof(int) * 2);
  const size_t total = off;

  gfh_plan* p = new (std::nothrow) gfh_plan();
  if (!p) return GFH_ERR_NOMEM;
  p->ctx = ctx;
  p->n_maps = n_maps;
  p->grids.assign(grids, grids + n_maps);
  p->cfg = tc;
  if (cudaSetDevice(ctx->device) != cudaSuccess) { delete p; return GFH_ERR_CUDA; }
  if (cudaMalloc(&p->d_buf, total) != cudaSuccess) { delete p; return GFH_ERR_NOMEM; }
  p->buf_bytes = total;
  char* base = (char*)p->d_buf;
  std::vector<char> h(total, 0);
  std::vector<MapDev> mds(n_maps);
  std::vector<int32_t> csr_map;
  csr_map.reserve(csr_entries);
  size_t key_off = 0;
  for (int m = 0; m < n_maps; ++m) {
    const gfh_grid& g = grids[m];
    HostMap& hm = hms[m];
    MapDev& md = mds[m];
    md.out = h_maps[m];
    md.UP = (const longlong2*)(base + o_U[m]);
    md.BS = (const longlong2*)(base + o_B[m]);
    md.col_band = (const int32_t*)(base + o_band[m]);
    md.f0c = (const double*)(base + o_f0[m]);
    md.f0n = (const double*)(base + o_f0n[m]);
    md.csr = (int64_t*)(base + o_csr[m]);
    md.keys = (unsigned long long*)(base + o_keys) + key_off;
    md.sums = md.keys + g.n_bands;
    key_off += g.n_bands + 2;
    md.cands = h_cands ? h_cands[m] : nullptr;
    md.stats = d_stats ? d_stats + m : nullptr;
    md.W = g.n_x0;
    md.ld = g.ld_x0;
    md.cells = hm.cells;
    md.x0_min = g.x0_min;
    md.dx0 = g.dx0;
    md.k_min = g.k_min;
    md.dk = g.dk;
    md.K = g.n_k;
    md.bin_lo = g.bin_lo;
    md.bin_hi = g.bin_hi;
    md.n_fft = g.n_fft;
    md.list = g.list;
    md.n_bands = g.n_bands;
    md.csr_base = (int32_t)csr_map.size();
    // paired tables: one 16-byte load per bin and one per FFT in the kernel
    int64_t* up = (int64_t*)(h.data() + o_U[m]);
    for (size_t j = 0; j + 1 < hm.U.size(); ++j) { up[2 * j] = hm.U[j + 1]; up[2 * j + 1] = hm.U[j]; }
    int64_t* bs = (int64_t*)(h.data() + o_B[m]);
    for (size_t i = 0; i < hm.B.size(); ++i) { bs[2 * i] = hm.B[i]; bs[2 * i + 1] = hm.S[i]; }
    std::memcpy(h.data() + o_band[m], hm.band.data(), sizeof(int32_t) * hm.band.size());
    std::memcpy(h.data() + o_f0[m], hm.f0.data(), sizeof(double) * hm.f0.size());
    std::memcpy(h.data() + o_f0n[m], hm.f0n.data(), sizeof(double) * hm.f0n.size());
    for (int e = 0; e < g.bin_hi - g.bin_lo + 2; ++e) csr_map.push_back(m);
  }
  std::memcpy(h.data() + o_maps, mds.data(), sizeof(MapDev) * n_maps);
  if (!tiles.empty()) std::memcpy(h.data() + o_tiles, tiles.data(), sizeof(TileDev) * tiles.size());
  std::memcpy(h.data() + o_csrmap, csr_map.data(), sizeof(int32_t) * csr_map.size());
  if (cudaMemcpy(p->d_buf, h.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    gfh_plan_destroy(p);
    return GFH_ERR_CUDA;
  }
  p->d_maps = (MapDev*)(base + o_maps);
  p->d_tiles = (TileDev*)(base + o_tiles);
  p->n_tiles = n_tiles_k;
  p->n_tiles_x = (int)tiles.size() - n_tiles_k;
  p->map_xd = map_xd;
  p->max_tile_bands = max_tile_bands;
  p->d_keys = (unsigned long long*)(base + o_keys);
  p->key_words = key_words;
  p->csr_entries = (int32_t)csr_entries;
  p->d_csr_map = (int32_t*)(base + o_csrmap);
  p->select = h_cands != nullptr || d_stats != nullptr;
  p->d_offsets_single = (int64_t*)(base + o_single);
  p->d_next = (int*)(base + o_next);
  p->h_maps.assign(h_maps, h_maps + n_maps);
  if (h_cands) p->h_cands.assign(h_cands, h_cands + n_maps);
  p->d_stats = d_stats;
  const int prc = gfh_prepare_plan(p);
  if (prc) {
    gfh_plan_destroy(p);
    return prc;
  }
  *out = p;
  return GFH_OK;
}

extern "C" int gfh_plan_execute(gfh_plan* p, const gfh_peaks* peaks) {
  if (!p || !peaks || !peaks->fft_idx || !peaks->bin || !peaks->offsets || peaks->n_lists < 1)
    return GFH_ERR_ARG;
  for (const gfh_grid& g : p->grids)
    if (g.list < 0 || g.list >= peaks->n_lists) return GFH_ERR_ARG;
  return gfh_launch_plan(p, peaks);
}

// ---- coarse tiles --------------------------------------------------------------------------------

extern "C" int gfh_plan_set_coarse(gfh_plan* p, int32_t coarse_k, int32_t coarse_x,
                                   int32_t max_sel) {
  if (!p || coarse_k < 1 || coarse_x < 1 || coarse_k > 4096 || coarse_x > 4096 || max_sel < 1 ||
      (int64_t)max_sel > (int64_t)coarse_k * coarse_x)
    return GFH_ERR_ARG;
  if (p->n_tiles_x > 0) return GFH_ERR_ARG;     // coarse tiles need lines moving <= 2 columns per row
  const int nct = coarse_k * coarse_x;
  std::vector<TileDev> fine;
  std::vector<int32_t> first;
  // the search's tile, chunk sums and band keys; the FFT sub-ranges fit in what the list kernel's
  // occupancy leaves
  const int sub_cap = sub_capacity((size_t)p->cfg.rows * (p->cfg.cols + 2) * 4 + 32 * 4 +
                                       (p->select ? (size_t)p->max_tile_bands * 8 + 64 : 0),
                                   p->cfg.threads);
  std::vector<CoarseMapDev> cms(p->n_maps);
  std::vector<size_t> fblk_off(p->n_maps);
  size_t fblk_total = 0;
  int n_lists = 0, fblk_entries = 0;
  first.reserve((size_t)p->n_maps * (nct + 1) + 1);
  int max_fine = 0, max_bands = p->max_tile_bands;
  size_t worst = 0;                        // longest gathered list: every map at its largest
  for (int m = 0; m < p->n_maps; ++m) {
    const gfh_grid& g = p->grids[m];
    HostMap hm;
    int rc = gfh_host_tables(&g, hm.U, hm.B, hm.S);
    if (rc) return rc;
    rc = gfh_host_columns(&g, hm.band, hm.f0, hm.f0n);
    if (rc) return rc;
    const size_t map_begin = fine.size();
    {
      CoarseMapDev& cm = cms[m];
      const int J = g.bin_hi - g.bin_lo + 1;
      cm.nb1 = (g.n_fft + kFftBlock - 1) / kFftBlock + 1;
      cm.list = g.list;
      cm.b0 = hm.B[0];
      cm.s0 = hm.S[0];
      cm.db = g.n_fft > 1 ? (double)(hm.B[g.n_fft - 1] - hm.B[0]) / (g.n_fft - 1) : 0.0;
      cm.ds = g.n_fft > 1 ? (double)(hm.S[g.n_fft - 1] - hm.S[0]) / (g.n_fft - 1) : 0.0;
      if ((int64_t)J * cm.nb1 > INT32_MAX) return GFH_ERR_SIZE;
      fblk_off[m] = fblk_total;
      fblk_total += (size_t)J * cm.nb1;
      fblk_entries = std::max(fblk_entries, J * cm.nb1);
      n_lists = std::max(n_lists, g.list + 1);
    }
    // columns of each f0 tile: analysis columns only; f0 falls with the column, so each range is
    // contiguous
    std::vector<int64_t> cmin(coarse_x, INT64_MAX), cmax(coarse_x, -1);
    const double span = g.ana_hi - g.ana_lo;
    for (int64_t c = 0; c < g.n_x0; ++c) {
      if (hm.band[c] < 0) continue;
      int xt = (int)std::floor((hm.f0[c] - g.ana_lo) / span * coarse_x);
      xt = std::min(std::max(xt, 0), coarse_x - 1);
      cmin[xt] = std::min(cmin[xt], c);
      cmax[xt] = std::max(cmax[xt], c);
    }
    std::vector<int> sizes;
    for (int kt = 0; kt < coarse_k; ++kt) {
      // rows r with floor(r coarse_k / K) = kt
      const int r0 = (int)(((int64_t)kt * g.n_k + coarse_k - 1) / coarse_k);
      const int r1 = (int)(((int64_t)(kt + 1) * g.n_k + coarse_k - 1) / coarse_k);
      for (int xt = 0; xt < coarse_x; ++xt) {
        first.push_back((int32_t)fine.size());
        const size_t before = fine.size();
        if (r1 > r0 && cmax[xt] >= 0) {
          // 16-byte aligned column range (vector stores): neighbouring tiles may share <= 3 columns
          const int64_t c_lo = cmin[xt] & ~int64_t(3);
          const int64_t c_hi = std::min<int64_t>(g.ld_x0, (cmax[xt] + 4) & ~int64_t(3));
          map_tiles(g, hm, m, p->cfg, r0, r1, c_lo, c_hi, fine, max_bands);
        }
        const int cnt = (int)(fine.size() - before);
        max_fine = std::max(max_fine, cnt);
        sizes.push_back(cnt);
      }
    }
    // group nct: the whole map, as gfh_plan_execute tiles it
    first.push_back((int32_t)fine.size());
    const size_t before = fine.size();
    map_tiles(g, hm, m, p->cfg, 0, g.n_k, 0, g.ld_x0, fine, max_bands);
    const size_t whole = fine.size() - before;
    for (size_t q = map_begin; q < fine.size(); ++q)
      fine[q].sub = tile_walks_sub_ranges(g, hm, fine[q], p->cfg.rows, sub_cap) ? 1 : 0;
    std::sort(sizes.begin(), sizes.end(), std::greater<int>());
    size_t top = 0;
    for (int i = 0; i < max_sel && i < (int)sizes.size(); ++i) top += sizes[i];
    worst += std::max(whole, top);
  }
  first.push_back((int32_t)fine.size());
  if (fine.size() > (size_t)INT32_MAX || worst > (size_t)INT32_MAX) return GFH_ERR_SIZE;
  if (max_bands > p->max_tile_bands + 8) {   // the sub-range room assumed the plan's band keys
    for (TileDev& t : fine) t.sub = 0;
  }
  const size_t smem = (size_t)p->cfg.rows * (p->cfg.cols + 2) * 4 + 32 * 4 +
                      (p->select ? (size_t)max_bands * 8 : 0) + (size_t)sub_cap * 8 + 16;
  if (smem > kHoughSmemLimit) return GFH_ERR_SIZE;

  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_fine = take(sizeof(TileDev) * std::max<size_t>(fine.size(), 1));
  const size_t o_first = take(sizeof(int32_t) * first.size());
  const size_t o_sel = take(sizeof(TileDev) * std::max<size_t>(worst, 1));
  const size_t o_cnt = take(2 * sizeof(int));
  const size_t o_cms = take(sizeof(CoarseMapDev) * p->n_maps);
  const size_t o_uns = take(sizeof(int) * std::max(n_lists, 1));
  const size_t o_fblk = take(sizeof(int32_t) * std::max<size_t>(fblk_total, 1));
  GFH_CUDA_TRY(cudaSetDevice(p->ctx->device));
  if (p->ctx->stream) GFH_CUDA_TRY(cudaStreamSynchronize(p->ctx->stream));
  void* buf = nullptr;
  if (cudaMalloc(&buf, off) != cudaSuccess) return GFH_ERR_NOMEM;
  char* base = (char*)buf;
  for (int m = 0; m < p->n_maps; ++m) cms[m].fblk = (int32_t*)(base + o_fblk) + fblk_off[m];
  cudaError_t e = cudaSuccess;
  if (!fine.empty())
    e = cudaMemcpy(base + o_fine, fine.data(), sizeof(TileDev) * fine.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(base + o_first, first.data(), sizeof(int32_t) * first.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(base + o_cms, cms.data(), sizeof(CoarseMapDev) * cms.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(buf); return GFH_ERR_CUDA; }
  if (p->d_coarse_buf) cudaFree(p->d_coarse_buf);
  p->d_coarse_buf = buf;
  p->d_fine = (TileDev*)(base + o_fine);
  p->d_coarse_first = (int32_t*)(base + o_first);
  p->d_sel_tiles = (TileDev*)(base + o_sel);
  p->d_sel_count = (int*)(base + o_cnt);
  p->sel_cap = (int)std::max<size_t>(worst, 1);
  p->coarse_k = coarse_k;
  p->coarse_x = coarse_x;
  p->max_sel = max_sel;
  p->max_fine = max_fine;
  p->max_tile_bands = max_bands;
  p->d_cmaps = (CoarseMapDev*)(base + o_cms);
  p->d_fft_unsorted = (int*)(base + o_uns);
  p->n_list_flags = std::max(n_lists, 1);
  p->sub_cap = sub_cap;
  p->fblk_entries = fblk_entries;
  p->n_sub_tiles = 0;
  for (const TileDev& t : fine) p->n_sub_tiles += t.sub;
  return GFH_OK;
}

extern "C" int gfh_plan_execute_tiles(gfh_plan* p, const gfh_peaks* peaks, const int32_t* d_coarse,
                                      int32_t n_sel, const int32_t* d_full) {
  if (!p || !peaks || !peaks->fft_idx || !peaks->bin || !peaks->offsets || peaks->n_lists < 1 ||
      p->coarse_k < 1 || n_sel < 0 || n_sel > p->max_sel || (n_sel > 0 && !d_coarse))
    return GFH_ERR_ARG;
  for (const gfh_grid& g : p->grids)
    if (g.list < 0 || g.list >= peaks->n_lists) return GFH_ERR_ARG;
  return gfh_launch_plan_tiles(p, peaks, d_coarse, n_sel, d_full);
}

// ---- autotuner ----------------------------------------------------------------------------------

namespace {

// Shapes the autotuner chose, by plan signature (plan_signature), for this process.
std::mutex g_tune_mu;
std::map<std::string, gfh_tile_config> g_tune_cache;

// Signature of a plan and its peak lists for the autotuner's cache: the device (compute capability,
// SMs), whether candidates are selected, and per map its k rows, x0 columns, bins, FFTs, line form
// (along k or along x0) and peak-density class: log2 of its list's peaks per (FFT, bin) of its
// band, in quarter steps (the list offsets are read back; the autotuner synchronises anyway).
int plan_signature(const gfh_plan* p, const gfh_peaks* peaks, std::string* key) {
  std::vector<int64_t> off((size_t)peaks->n_lists + 1);
  if (p->ctx->stream) GFH_CUDA_TRY(cudaStreamSynchronize(p->ctx->stream));
  GFH_CUDA_TRY(cudaMemcpy(off.data(), peaks->offsets, off.size() * sizeof(int64_t),
                          cudaMemcpyDeviceToHost));
  cudaDeviceProp prop{};
  GFH_CUDA_TRY(cudaGetDeviceProperties(&prop, p->ctx->device));
  std::string k = "cc" + std::to_string(prop.major) + "." + std::to_string(prop.minor) + " sm" +
                  std::to_string(prop.multiProcessorCount) + (p->select ? " sel" : " nosel");
  for (int m = 0; m < p->n_maps; ++m) {
    const gfh_grid& g = p->grids[m];
    if (g.list < 0 || g.list >= peaks->n_lists) return GFH_ERR_ARG;
    const double cells = (double)g.n_fft * (double)(g.bin_hi - g.bin_lo + 1);
    const double n = (double)(off[g.list + 1] - off[g.list]);
    const int cls = n > 0.0 ? (int)std::floor(4.0 * std::log2(n / cells)) : -1000;
    k += " " + std::to_string(g.n_k) + "x" + std::to_string(g.n_x0) + "b" +
         std::to_string(g.bin_hi - g.bin_lo + 1) + "f" + std::to_string(g.n_fft) +
         (p->map_xd[m] ? "x" : "k") + "d" + std::to_string(cls);
  }
  *key = k;
  return GFH_OK;
}

// Mean time of `reps` executions of plan q on its stream (after one untimed run), in ms.
int time_plan(gfh_plan* q, const gfh_peaks* peaks, int reps, float* ms) {
  cudaStream_t st = q->ctx->stream;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return GFH_ERR_CUDA;
  }
  int rc = gfh_plan_execute(q, peaks);
  if (!rc && cudaEventRecord(a, st) != cudaSuccess) rc = GFH_ERR_CUDA;
  for (int i = 0; i < reps && !rc; ++i) rc = gfh_plan_execute(q, peaks);
  if (!rc && cudaEventRecord(b, st) != cudaSuccess) rc = GFH_ERR_CUDA;
  if (!rc && cudaEventSynchronize(b) != cudaSuccess) rc = GFH_ERR_CUDA;
  if (!rc && cudaEventElapsedTime(ms, a, b) != cudaSuccess) rc = GFH_ERR_CUDA;
  if (!rc) *ms /= (float)reps;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

// Rebuilds plan p with tile shape `shape` (same grids and outputs; coarse tiles follow the shape).
bool same_shape(const gfh_tile_config& a, const gfh_tile_config& b) {
  return a.rows == b.rows && a.cols == b.cols && a.threads == b.threads && a.form == b.form;
}

int reshape_plan(gfh_plan* p, const gfh_tile_config& shape) {
  if (same_shape(shape, p->cfg)) return GFH_OK;
  gfh_plan* q = nullptr;
  gfh_tile_config cfg = shape;
  int rc = gfh_plan_create(p->ctx, p->n_maps, p->grids.data(), p->h_maps.data(),
                           p->h_cands.empty() ? nullptr : p->h_cands.data(), p->d_stats, &cfg, &q);
  if (rc) return rc;
  if (p->ctx->stream) cudaStreamSynchronize(p->ctx->stream);
  const int ck = p->coarse_k, cx = p->coarse_x, ms = p->max_sel;
  std::swap(*p, *q);      // p takes the new tables; q holds the old ones and is freed
  gfh_plan_destroy(q);
  if (ck > 0) return gfh_plan_set_coarse(p, ck, cx, ms);
  return GFH_OK;
}

}  // namespace

extern "C" int gfh_plan_autotune(gfh_plan* p, const gfh_peaks* peaks, int32_t reps,
                                 gfh_tile_config* h_best, float* h_best_ms) {
  if (!p || !peaks || !peaks->offsets || peaks->n_lists < 1 || reps < 1) return GFH_ERR_ARG;
  static const int kRowsList[] = {4, 8, 16};
  static const int kColsList[] = {1024, 2048, 3072, 4096};
  static const int kThreadsList[] = {256, 512, 1024};
  std::string key;
  int rc = plan_signature(p, peaks, &key);
  if (rc) return rc;
  bool cached = false;
  gfh_tile_config best = p->cfg;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) { best = it->second; cached = true; }
  }
  float best_ms = 0.f;
  if (cached) {                 // tuned before: take that shape and time it alone
    rc = reshape_plan(p, best);
    if (!rc) rc = time_plan(p, peaks, reps, &best_ms);
    if (rc) return rc;
    if (h_best) *h_best = best;
    if (h_best_ms) *h_best_ms = best_ms;
    return GFH_OK;
  }
  rc = time_plan(p, peaks, reps, &best_ms);
  if (rc) return rc;
  auto try_shape = [&](const gfh_tile_config& cfg) -> int {
    if (same_shape(cfg, p->cfg)) return GFH_OK;
    gfh_plan* q = nullptr;
    gfh_tile_config c = cfg;
    const int crc = gfh_plan_create(p->ctx, p->n_maps, p->grids.data(), p->h_maps.data(),
                                    p->h_cands.empty() ? nullptr : p->h_cands.data(), p->d_stats,
                                    &c, &q);
    if (crc == GFH_ERR_SIZE || crc == GFH_ERR_ARG) return GFH_OK;   // shape does not fit
    if (crc) return crc;
    float ms = 0.f;
    const int trc = time_plan(q, peaks, reps, &ms);
    gfh_plan_destroy(q);
    if (trc) return trc;
    if (ms < best_ms) { best_ms = ms; best = cfg; }
    return GFH_OK;
  };
  for (int r : kRowsList)
    for (int c : kColsList)
      for (int t : kThreadsList) {
        if (t == 1024 && r < 16) continue;     // 1024 threads only for 16-row tiles
        rc = try_shape(gfh_tile_config{r, c, t, 0});
        if (rc) return rc;
      }
  // the fastest shape with the other drawing form
  gfh_tile_config other = best;
  other.form = 1 - best.form;
  rc = try_shape(other);
  if (rc) return rc;
  rc = reshape_plan(p, best);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  if (h_best) *h_best = best;
  if (h_best_ms) *h_best_ms = best_ms;
  return GFH_OK;
}

extern "C" int gfh_autotune_cache_size(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tune_cache.size();
}

extern "C" void gfh_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
}
